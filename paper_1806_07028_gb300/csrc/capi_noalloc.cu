// pcamg_residual_noalloc: the fine-level residual r = b - A x with ||r||^2, for
// callers that must not allocate device memory.
//
// Who needs this: code that runs where a device allocation is not allowed or
// not wanted -- for instance a time-critical loop that may not pay for
// cudaMalloc/cudaFree (which can synchronise the whole device), or a process
// whose device memory is entirely handed out by its own pool. Those callers
// pass only their inputs and outputs; the per-block partial sums of ||r||^2
// live in a fixed array below instead of a buffer allocated per call.
//
// The array is a file-scope __device__ variable: every GPU that loads this
// library holds it (kNoAllocPartials doubles) until the process exits. Host
// code may not use its name as a device pointer; the device address is looked
// up once per device with cudaGetSymbolAddress (with that device current) on
// the first call made on that device, and cached for the life of the process,
// which assumes the device's primary context is not reset in between. The
// launch shape depends on n alone, so a call reads nothing back and does not
// synchronise: it returns once the work is queued on the stream.
#include <mutex>

#include "pcamg_internal.cuh"

namespace {

// one partial per block of the norm launch (1,024 rows each): at most 65,536
// blocks, n <= 67,108,864 rows
constexpr int kNoAllocPartials = 65536;
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_partials[kNoAllocPartials];

std::mutex g_noalloc_mu;
double* g_noalloc_ptr[kNoAllocMaxDevices] = {nullptr};

pcamg_status noalloc_fail(pcamg_status s, const char* msg) {
    pc::set_global_error(msg);   // readable through pcamg_last_error(NULL)
    return s;
}

}  // namespace

extern "C" {

PCAMG_API pcamg_status pcamg_residual_noalloc(int32_t n, const int32_t* d_rowptr,
                                              const int32_t* d_col, const double* d_val,
                                              const double* d_x, const double* d_b,
                                              double* d_r, double* d_norm2, void* stream) {
    if (n < 1 || !d_rowptr || !d_col || !d_val || !d_x || !d_b || !d_r || !d_norm2)
        return noalloc_fail(PCAMG_ERR_INVALID, "pcamg_residual_noalloc: invalid argument");
    if (pc::residual_norm_blocks(n) > kNoAllocPartials)
        return noalloc_fail(PCAMG_ERR_INVALID,
                            "pcamg_residual_noalloc: n exceeds 67,108,864 rows (fixed scratch size)");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) {
        cudaGetLastError();
        return noalloc_fail(PCAMG_ERR_CUDA, "pcamg_residual_noalloc: no usable current device");
    }
    double* partials = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                return noalloc_fail(PCAMG_ERR_CUDA, "pcamg_residual_noalloc: cudaGetSymbolAddress failed");
            }
            g_noalloc_ptr[dev] = static_cast<double*>(p);
        }
        partials = g_noalloc_ptr[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    try {
        // with ||r||^2 requested the residual runs the streaming kernel, whose
        // launch depends on n only (no nnz, no lanes per row)
        pc::Csr A;
        A.n = n;
        A.rowptr = d_rowptr;
        A.col = d_col;
        A.val = d_val;
        // every block writes its own partial, so nothing needs clearing
        pc::residual64(s, A, d_x, d_b, d_r, partials, d_norm2);   // checks the launch
    } catch (const pc::Error& e) {
        pc::set_global_error(e.msg);
        return e.status;
    }
    return PCAMG_OK;
}

}  // extern "C"
