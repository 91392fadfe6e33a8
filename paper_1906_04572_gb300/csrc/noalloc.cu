// corutv_orth_noalloc: the thin QR of corutv_orth (CholeskyQR2 with the
// shifted fallback pass) for callers that must not allocate device memory.
//
// Who needs this: code that runs where cudaMalloc is not allowed or not
// wanted -- a host framework that owns every byte of device memory through
// its own pool, a real-time or safety-certified process that forbids
// allocation after start-up, or a plug-in called from inside another
// library's step that may not grow memory behind that library's back. Such
// callers pass their inputs and outputs and nothing else.
//
// How: all temporaries live in one file-scope __device__ array of
// kScratchBytes (16 MiB). Every GPU that loads this library holds that array
// until the process exits. Host code cannot pass the array's name to a
// kernel (in host code it is only a stand-in symbol), so on its first call
// on a device this entry point, with that device current, asks the runtime
// for the array's device address once (cudaGetSymbolAddress) and caches it.
// Make that first call on each device before any stream capture begins.
//
// All calls share the one array and it keeps the previous call's contents:
// the status words are cleared at the start of every call, everything else
// is fully overwritten before it is read. Calls that overlap on the GPU
// (different streams, or different host threads without ordering) race on
// the array and corrupt each other's results; order them on one stream.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "../../include/corutv.h"
#include "internal.cuh"

namespace {

constexpr size_t kScratchBytes = size_t(16) << 20;
constexpr int64_t kMaxPanelElems = int64_t(1) << 19;  // round_up(rows, 64) * ell
constexpr int kMaxGramSplits = 16;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

void* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;
// Failures are reported by status; the message is readable through
// corutv_last_error() from the calling thread.
corutv_status noalloc_fail(corutv_status st, const char* msg, cudaError_t e = cudaSuccess) {
    char buf[384];
    if (e != cudaSuccess) snprintf(buf, sizeof(buf), "corutv_orth_noalloc: %s: %s", msg, cudaGetErrorString(e));
    else snprintf(buf, sizeof(buf), "corutv_orth_noalloc: %s", msg);
    corutv::record_error(buf);
    return st;
}

int64_t rup(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

// Device (or managed) memory, asked of the runtime (no allocation). A host
// pointer passed by mistake would otherwise reach the kernels as a raw address.
bool on_device(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

extern "C" corutv_status corutv_orth_noalloc(const double* C, int64_t rows, int64_t ell, int64_t ldc, double* Q,
                                            int64_t ldq, double* R, int* info, void* cuda_stream) {
    using namespace corutv;
    if (!C || !Q) return noalloc_fail(CORUTV_EINVAL, "C and Q must not be NULL");
    if (!on_device(C) || !on_device(Q) || (R && !on_device(R)) || (info && !on_device(info)))
        return noalloc_fail(CORUTV_EINVAL, "C, Q, R and info must be device memory");
    if (ell < 1 || ell > 128 || rows < ell || ldc < ell || ldq < ell)
        return noalloc_fail(CORUTV_EINVAL, "need 1 <= ell <= 128, rows >= ell, ldc >= ell, ldq >= ell");
    const int64_t ld = rup(rows, 64);
    if (ld * ell > kMaxPanelElems)
        return noalloc_fail(CORUTV_EINVAL,
                            "rows x ell too large for the fixed 16 MiB scratch: need round_up(rows, 64) * ell "
                            "<= 524288 (for example 4096 x 128)");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(CORUTV_ECUDA, "cudaGetDevice failed", e);
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(CORUTV_EINVAL, "device index out of range");
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_scratch_mu);
        if (!g_scratch_addr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p)
                return noalloc_fail(CORUTV_ECUDA, "cudaGetSymbolAddress of the scratch array failed", e);
            g_scratch_addr[dev] = p;
        }
        base = g_scratch_addr[dev];
    }
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return noalloc_fail(CORUTV_ECUDA, "cudaDeviceGetAttribute failed", e);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);

    // carve the scratch: three panels, Gram partials, G, R, status words
    unsigned char* sp = static_cast<unsigned char*>(base);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        unsigned char* p = sp + off;
        off += align256(bytes);
        return p;
    };
    const size_t panel = sizeof(double) * (size_t)(ld * ell);
    double* cp = reinterpret_cast<double*>(take(panel));
    double* qp = reinterpret_cast<double*>(take(panel));
    double* tp = reinterpret_cast<double*>(take(panel));
    int gs = gemm_simt_splits(ell, rows, sms);
    if (gs > kMaxGramSplits) gs = kMaxGramSplits;
    double* gpart = reinterpret_cast<double*>(take(sizeof(double) * (size_t)(gs * ell * ell)));
    double* g = reinterpret_cast<double*>(take(sizeof(double) * (size_t)(ell * ell)));
    double* r = reinterpret_cast<double*>(take(sizeof(double) * (size_t)(ell * ell)));
    int* flags = reinterpret_cast<int*>(take(sizeof(int) * FLAG_COUNT));
    int* skip = reinterpret_cast<int*>(take(sizeof(int) * 8));
    if (off > kScratchBytes) return noalloc_fail(CORUTV_EINVAL, "internal: scratch layout exceeds 16 MiB");

    // status words start at zero on every call
    e = cudaMemsetAsync(flags, 0, sizeof(int) * FLAG_COUNT, st);
    if (e != cudaSuccess) return noalloc_fail(CORUTV_ECUDA, "cudaMemsetAsync failed", e);

    auto gram = [&](const double* x, const double* y, const int* cancel) -> cudaError_t {
        const int64_t ll = ell * ell;
        GemmArgs ga{A_PANEL_T, B_PANEL, O_ROWMAJ, T_F64, T_F64, x, ld, y, ld, gpart, ell, ll,
                    ell, rows, ell, gs, cancel};
        cudaError_t ee = launch_gemm_simt(ga, st);
        if (ee != cudaSuccess) return ee;
        return launch_reduce_splits(gpart, T_F64, gs, ll, g, T_F64, ell, ell, ell, ell, cancel, st);
    };
#define NA_CK(expr)                                                                       \
    do {                                                                                  \
        cudaError_t ee_ = (expr);                                                         \
        if (ee_ != cudaSuccess) return noalloc_fail(CORUTV_ECUDA, #expr " failed", ee_);  \
    } while (0)
    NA_CK(launch_rowmajor_to_panel(C, ldc, rows, ell, ell, cp, T_F64, ld, st));
    // pass 1 (shifted when the Gram is not numerically positive definite)
    NA_CK(gram(cp, cp, nullptr));
    NA_CK(launch_cholesky(g, ell, rows, r, flags, skip, nullptr, st));
    NA_CK(launch_trsm_rows(cp, T_F64, ld, rows, ell, r, T_F64, tp, ld, nullptr, T_F64, 0, nullptr, st));
    // pass 1b, only after a shifted pass 1
    NA_CK(gram(tp, tp, skip));
    NA_CK(launch_cholesky(g, ell, rows, r, flags, nullptr, skip, st));
    NA_CK(launch_trsm_rows(tp, T_F64, ld, rows, ell, r, T_F64, tp, ld, nullptr, T_F64, 0, skip, st));
    // pass 2
    NA_CK(gram(tp, tp, nullptr));
    NA_CK(launch_cholesky(g, ell, rows, r, flags, nullptr, nullptr, st));
    NA_CK(launch_trsm_rows(tp, T_F64, ld, rows, ell, r, T_F64, qp, ld, nullptr, T_F64, 0, nullptr, st));
    NA_CK(launch_panel_to_rowmajor(qp, ld, rows, ell, Q, T_F64, ldq, nullptr, st));
    if (R) {
        // R = Q^T C, upper triangular in exact arithmetic
        NA_CK(gram(qp, cp, nullptr));
        NA_CK(cudaMemcpyAsync(R, g, sizeof(double) * (size_t)(ell * ell), cudaMemcpyDeviceToDevice, st));
    }
    if (info) NA_CK(cudaMemcpyAsync(info, flags + FLAG_BREAKDOWN, sizeof(int), cudaMemcpyDeviceToDevice, st));
#undef NA_CK
    return CORUTV_OK;
}
