// Exact assignment that allocates no device memory.
//
// For callers that may not allocate device memory themselves or let a
// library do it: a process whose device memory is all owned by another
// framework's fixed pool, or a long-running service that must not allocate
// after start-up.  The scratch (pair distances, counters) is one file-scope
// __device__ array of fixed size that every GPU which loads this library
// keeps until the process exits.  The paper has no counterpart; it is the
// same computation as d2_assign without a pruner.
#include <algorithm>
#include <mutex>

#include "d2_internal.cuh"

// 256 bytes of counters followed by D2_NOALLOC_MAX_PAIRS pair distances
#define D2_NOALLOC_HEAD 64
static __device__ __align__(256) float g_noalloc_scratch[D2_NOALLOC_HEAD + D2_NOALLOC_MAX_PAIRS];

int d2_assign_exact_into(const d2_bags* b, int K, int m, const float* x, const float* w, int32_t* labels,
                         float* dist, float* D, int* flags, int64_t* fail_count, int device, cudaStream_t st,
                         cudaError_t* cerr);

#define D2_NOALLOC_MAX_DEVICES 64
static float* g_scratch_addr[D2_NOALLOC_MAX_DEVICES];
static std::mutex g_scratch_mu;

// Device address of the scratch array on the current device, resolved once
// per device (the symbol's name in host code is only a host-side handle).
// The cached address is not refreshed after cudaDeviceReset (the header says
// so: the entry point must not be used after a reset).
static cudaError_t scratch_on(int device, float** out) {
    if (device < 0 || device >= D2_NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[device] = static_cast<float*>(p);
    }
    *out = g_scratch_addr[device];
    return cudaSuccess;
}

extern "C" int d2_assign_noalloc(const d2_bags* bags, int32_t K, int32_t m, const float* x, const float* w,
                                 int32_t* labels, float* dist, void* stream) {
    if (!bags || !x || !w || !labels || !dist || K < 1 || m < 1) return D2_EINVAL;
    if (bags->N < 1 || bags->n < 1 || bags->d < 1 || bags->max_mk < 1 || !bags->offsets || !bags->wt)
        return D2_EINVAL;
    if ((bags->supp != nullptr) == (bags->vocab_idx != nullptr && bags->vocab != nullptr)) return D2_EINVAL;
    if (bags->N * (int64_t)K > D2_NOALLOC_MAX_PAIRS) return D2_ESCRATCH;
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) return D2_ECUDA;
    float* scratch = nullptr;
    if (scratch_on(device, &scratch) != cudaSuccess) return D2_ECUDA;
    cudaStream_t st = d2_stream(stream);
    // the array keeps the previous call's contents: clear the counters
    if (cudaMemsetAsync(scratch, 0, D2_NOALLOC_HEAD * sizeof(float), st) != cudaSuccess) return D2_ECUDA;
    int* flags = reinterpret_cast<int*>(scratch);
    int64_t* fails = reinterpret_cast<int64_t*>(scratch + 2);
    float* D = scratch + D2_NOALLOC_HEAD;
    cudaError_t ce = cudaSuccess;
    const int rc = d2_assign_exact_into(bags, K, m, x, w, labels, dist, D, flags, fails, device, st, &ce);
    if (rc) return rc;
    // a pair that reached the solver's phase cap leaves a wrong W^2 and label:
    // read the count back (this makes the call synchronous)
    int64_t nfail = 0;
    if (cudaMemcpyAsync(&nfail, fails, sizeof(nfail), cudaMemcpyDeviceToHost, st) != cudaSuccess) return D2_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return D2_ECUDA;
    return nfail > 0 ? D2_ENOCONV : D2_OK;
}
