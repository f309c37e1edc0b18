// Rotation-pair selection that allocates no device memory.
//
// Some callers cannot call cudaMalloc: code that runs inside another
// framework's memory pool, under a strict device-memory budget fixed at start,
// or in a process where the allocator is owned by someone else. This entry
// point gives them the occupied-virtual pair selection of a sweep (|F_ij| >= tau,
// at most k_max of the largest, ties at the cut kept) on arrays they already
// own. Its working memory is a file-scope __device__ array: every GPU that
// loads the library holds it (kNoallocScratchBytes) until the process exits.
#include <cuda.h>

#include <algorithm>
#include <mutex>

#include "sscf_internal.h"

namespace {

constexpr long long kNoallocMaxValues = 1ll << 21;   // largest n accepted
constexpr int kHdr = 288;                            // header words (histogram + state)
// header layout (64-bit words): [0, 256) histogram, 256 candidates, 257 prefix,
// 258 mask, 259 rank still to find, 260 threshold key, 261 kept pairs
constexpr int kCand = 256, kPrefix = 257, kMask = 258, kRank = 259, kThr = 260, kKept = 261;

// Scratch of the no-allocation path: a header, then the candidate keys.
// Calls share it and it keeps the last call's contents; each call clears the
// header first. Two calls that overlap on the GPU (different streams, or
// different host threads) race on it.
__device__ __align__(256) unsigned long long g_noalloc_scratch[kHdr + kNoallocMaxValues];
constexpr size_t kNoallocScratchBytes = sizeof(unsigned long long) * (kHdr + kNoallocMaxValues);

static_assert(kNoallocScratchBytes == 16 * 1024 * 1024 + 288 * 8, "scratch size stated in sscf.h");

std::mutex g_setup_mutex;
void* g_scratch_ptr[64] = {nullptr};
CUcontext g_scratch_ctx[64] = {nullptr};   // context the address was looked up in

__device__ __forceinline__ unsigned long long key_of(double v) {
    return (unsigned long long)__double_as_longlong(v);
}

__global__ void k_na_clear(unsigned long long* s) {
    for (int i = threadIdx.x; i < kHdr; i += blockDim.x) s[i] = 0ull;
}

__global__ void k_na_candidates(const double* __restrict__ f, long long n, double tau, unsigned long long* s) {
    unsigned long long* cand = s + kHdr;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double v = fabs(f[i]);
        if (v >= tau && v > 0.0) {
            const unsigned long long pos = atomicAdd(&s[kCand], 1ull);
            cand[pos] = key_of(v);
        }
    }
}

__global__ void k_na_hist(int shift, long long k_max, unsigned long long* s) {
    const unsigned long long nc = s[kCand];
    if (nc <= (unsigned long long)k_max) return;
    __shared__ unsigned h[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0u;
    __syncthreads();
    const unsigned long long prefix = s[kPrefix], mask = s[kMask];
    const unsigned long long* cand = s + kHdr;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < nc;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long k = cand[i];
        if ((k & mask) == prefix) atomicAdd(&h[(k >> shift) & 255ull], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += blockDim.x)
        if (h[i]) atomicAdd(&s[i], (unsigned long long)h[i]);
}

__global__ void k_na_pick(int shift, long long k_max, unsigned long long* s) {
    if (s[kCand] <= (unsigned long long)k_max) return;
    if (shift == 56) s[kRank] = (unsigned long long)k_max;
    unsigned long long k = s[kRank], cum = 0;
    int b = 255;
    for (; b > 0; --b) {
        if (cum + s[b] >= k) break;
        cum += s[b];
    }
    s[kPrefix] |= (unsigned long long)b << shift;
    s[kMask] |= 255ull << shift;
    s[kRank] = k - cum;
    for (int i = 0; i < 256; ++i) s[i] = 0ull;
    if (shift == 0) s[kThr] = s[kPrefix];
}

__global__ void k_na_mark(const double* __restrict__ f, long long n, double tau, unsigned char* __restrict__ keep,
                          unsigned long long* s) {
    const unsigned long long thr = s[kThr];
    unsigned long long kept = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double v = fabs(f[i]);
        const bool k = v >= tau && v > 0.0 && key_of(v) >= thr;
        keep[i] = k ? 1 : 0;
        kept += k ? 1 : 0;
    }
    for (int off = 16; off > 0; off >>= 1) kept += __shfl_xor_sync(0xffffffffu, kept, off);
    if ((threadIdx.x & 31) == 0 && kept) atomicAdd(&s[kKept], kept);
}

// The CUDA context current on this thread (driver entry point through the
// runtime, so the library needs no link to the driver library); NULL when
// none is current yet or the lookup is unavailable.
CUcontext current_context() {
    using GetCurrentFn = CUresult (*)(CUcontext*);
    static GetCurrentFn fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
        return (GetCurrentFn)p;
    }();
    CUcontext c = nullptr;
    if (!fn || fn(&c) != CUDA_SUCCESS) return nullptr;
    return c;
}

// Set-up, once per device, with that device current: the device address of
// the scratch array (in host code its name is only a stand-in, not a device
// address). The address belongs to the device's context: after a reset of
// that context (cudaDeviceReset) the module is loaded again, so the address is
// looked up again whenever the current context is not the one it came from.
int scratch_for_current_device(unsigned long long** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return SSCF_ERR_CUDA;
    }
    CUcontext cur = current_context();
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev] || cur == nullptr || cur != g_scratch_ctx[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return SSCF_ERR_CUDA;
        }
        g_scratch_ptr[dev] = p;
        g_scratch_ctx[dev] = current_context();   // current now: the lookup made it so
    }
    *out = (unsigned long long*)g_scratch_ptr[dev];
    return SSCF_OK;
}

}  // namespace

extern "C" int sscf_select_pairs_noalloc(const double* f, int64_t n, double tau, int64_t k_max,
                                         unsigned char* keep, int64_t* n_keep, void* cuda_stream) {
    if (n < 0 || k_max < 1 || !(tau >= 0.0)) return SSCF_ERR_INVALID_ARG;
    if (n > kNoallocMaxValues) return SSCF_ERR_INVALID_ARG;
    if (n > 0 && (!f || !keep)) return SSCF_ERR_INVALID_ARG;
    unsigned long long* s = nullptr;
    int st = scratch_for_current_device(&s);
    if (st != SSCF_OK) return st;
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    const int th = 256;
    const int blocks = (int)std::min<long long>((n + th - 1) / th + 1, 4096);
    k_na_clear<<<1, 256, 0, stream>>>(s);
    if (n > 0) {
        k_na_candidates<<<blocks, th, 0, stream>>>(f, n, tau, s);
        for (int shift = 56; shift >= 0; shift -= 8) {
            k_na_hist<<<std::min(blocks, 1024), th, 0, stream>>>(shift, k_max, s);
            k_na_pick<<<1, 1, 0, stream>>>(shift, k_max, s);
        }
        k_na_mark<<<blocks, th, 0, stream>>>(f, n, tau, keep, s);
    }
    if (cudaGetLastError() != cudaSuccess) return SSCF_ERR_CUDA;
    if (n_keep) {
        unsigned long long kept = 0;
        if (cudaMemcpyAsync(&kept, s + kKept, sizeof(kept), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
            cudaStreamSynchronize(stream) != cudaSuccess) {
            cudaGetLastError();
            return SSCF_ERR_CUDA;
        }
        *n_keep = (int64_t)kept;
    }
    return SSCF_OK;
}
