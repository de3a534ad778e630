// Allocation-free validation entry point.
//
// Some callers cannot allocate device memory when they need a validation:
// code that runs while a CUDA graph is being captured (cudaMalloc is not
// allowed there), latency-critical serving loops that must not call
// cudaMalloc/cudaFree because those calls can synchronize the device and
// stall every other stream, and plug-ins hosted by a framework that owns all
// device memory and gives them only their inputs and outputs.  For them this
// file provides hetm_validate_noalloc: the same per-tuple conflict test as
// hetm_validate_only, needing no context, whose only scratch memory is the
// file-scope array below.
//
// Scratch: one partial hit count and one error flag per block, in a static
// __device__ array that every GPU loading this library holds until the
// process exits.  Each block handles a fixed 8192-tuple span and writes its
// own slot; a one-block finalize kernel adds the slots up.  The count is an
// integer sum, so it does not depend on the order in which the slots are
// added.  The span and slot count bound the input to HETM_NOALLOC_MAX_TUPLES
// tuples.

#include <mutex>

#include "hetm_internal.cuh"

namespace {

constexpr uint64_t kSpan = 8192;  // tuples per block
constexpr uint32_t kSlots = HETM_NOALLOC_MAX_TUPLES / kSpan;
static_assert(kSlots * kSpan == HETM_NOALLOC_MAX_TUPLES, "slot count must divide the limit");

struct NoAllocScratch {
    unsigned long long hits[kSlots];
    int err[kSlots];
};

// The shared scratch of every hetm_validate_noalloc call on a device.
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

__device__ __forceinline__ uint4 ld_nc16(const void *p) {
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

__device__ __forceinline__ uint32_t rs_bit_of(const uint32_t *rs, uint32_t a, uint32_t gshift) {
    const uint32_t g = a >> gshift;
    return (__ldg(rs + (g >> 5)) >> (g & 31)) & 1u;
}

// Block b tests tuples [b * kSpan, min(n, (b + 1) * kSpan)) against RS_bmp;
// flags are bit-packed in log order (bit i of word i / 32) as in
// hetm_validate_only, and the block's hit count goes to its scratch slot.
__global__ void __launch_bounds__(256) k_validate_noalloc(const hetm_log_entry *__restrict__ log,
                                                          uint64_t n, const uint32_t *__restrict__ rs,
                                                          uint32_t gshift, uint64_t n_words,
                                                          uint32_t *__restrict__ flags,
                                                          NoAllocScratch *scr) {
    __shared__ unsigned long long s_hits[8];
    __shared__ int s_err;
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_err = 0;
    __syncthreads();
    const uint64_t lo = blockIdx.x * kSpan;
    const uint64_t hi = lo + kSpan < n ? lo + kSpan : n;
    uint32_t hits = 0;
    bool bad = false;
    // whole 128-tuple tiles: lane l holds tuples 4l..4l+3 as three 16-byte vectors
    const uint64_t full_hi = lo + ((hi - lo) / 128) * 128;
    for (uint64_t t0 = lo + warp * 128ull; t0 < full_hi; t0 += 8 * 128ull) {
        const char *p = reinterpret_cast<const char *>(log + t0) + lane * 48u;
        const uint4 q0 = ld_nc16(p), q1 = ld_nc16(p + 16), q2 = ld_nc16(p + 32);
        const uint32_t a[4] = {q0.x, q0.w, q1.z, q2.y};
        uint32_t nib = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (a[j] < n_words) nib |= rs_bit_of(rs, a[j], gshift) << j;
            else bad = true;
        }
        hits += __popc(nib);
        uint32_t w = nib << (4u * (lane & 7u));
        w |= __shfl_xor_sync(hetm::kFull, w, 1);
        w |= __shfl_xor_sync(hetm::kFull, w, 2);
        w |= __shfl_xor_sync(hetm::kFull, w, 4);
        if (flags && (lane & 7u) == 0) flags[t0 / 32 + (lane >> 3)] = w;
    }
    // ragged end of the input (only the last block): 32 tuples per warp step
    for (uint64_t e0 = full_hi + warp * 32ull; e0 < hi; e0 += 8 * 32ull) {
        const uint64_t i = e0 + lane;
        uint32_t bit = 0;
        if (i < hi) {
            const uint32_t a = log[i].addr;
            if (a < n_words) bit = rs_bit_of(rs, a, gshift);
            else bad = true;
        }
        const uint32_t w = __ballot_sync(hetm::kFull, bit);
        hits += bit;
        if (flags && lane == 0) flags[e0 / 32] = w;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) hits += __shfl_xor_sync(hetm::kFull, hits, o);
    if (lane == 0) s_hits[warp] = hits;
    if (bad) s_err = 1;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long sum = 0;
        for (int k = 0; k < 8; ++k) sum += s_hits[k];
        scr->hits[blockIdx.x] = sum;  // every slot of the grid is overwritten
        scr->err[blockIdx.x] = s_err;
    }
}

// Add up the first n_blocks slots into the caller's outputs (integer sums
// and ORs: the result does not depend on the order of the additions).
__global__ void __launch_bounds__(1024) k_noalloc_finish(const NoAllocScratch *scr,
                                                         uint32_t n_blocks,
                                                         unsigned long long *count, int *err) {
    __shared__ unsigned long long s_sum[32];
    __shared__ int s_err[32];
    unsigned long long sum = 0;
    int e = 0;
    for (uint32_t b = threadIdx.x; b < n_blocks; b += blockDim.x) {
        sum += scr->hits[b];
        e |= scr->err[b];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sum += __shfl_xor_sync(hetm::kFull, sum, o);
        e |= __shfl_xor_sync(hetm::kFull, e, o);
    }
    if ((threadIdx.x & 31) == 0) {
        s_sum[threadIdx.x >> 5] = sum;
        s_err[threadIdx.x >> 5] = e;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        int te = 0;
        for (unsigned k = 0; k < (blockDim.x + 31) / 32; ++k) {
            t += s_sum[k];
            te |= s_err[k];
        }
        *count = t;
        if (err) *err = te ? HETM_EDEVICE : HETM_OK;
    }
}

// Device address of g_noalloc_scratch, looked up once per device.
constexpr int kMaxDevices = 64;
std::mutex g_sym_mu;
void *g_sym_ptr[kMaxDevices] = {};

int scratch_for_current_device(NoAllocScratch **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return HETM_ECUDA;
    std::lock_guard<std::mutex> g(g_sym_mu);
    if (!g_sym_ptr[dev]) {
        void *p = nullptr;
        // the lookup's own return code decides; an error some earlier call
        // left pending on this thread is neither read nor cleared here
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return HETM_ECUDA;
        g_sym_ptr[dev] = p;
    }
    *out = static_cast<NoAllocScratch *>(g_sym_ptr[dev]);
    return HETM_OK;
}

bool is_pow2(uint64_t v) { return v && !(v & (v - 1)); }

}  // namespace

extern "C" int hetm_validate_noalloc(const hetm_log_entry *dev_log, uint64_t n,
                                     const uint32_t *dev_rs_bmp, uint32_t granule_bytes,
                                     uint64_t stmr_words, uint32_t *dev_flag_bits,
                                     uint64_t *dev_n_conflicts, int32_t *dev_err, void *stream) {
    if (n > HETM_NOALLOC_MAX_TUPLES) return HETM_ECAPACITY;
    if (!dev_n_conflicts || (n && (!dev_log || !dev_rs_bmp)) || !is_pow2(granule_bytes) ||
        granule_bytes < 4 || stmr_words == 0 || stmr_words >= (1ull << 32) ||
        (reinterpret_cast<uintptr_t>(dev_log) & 15))
        return HETM_EINVAL;
    NoAllocScratch *scr = nullptr;
    int rc = scratch_for_current_device(&scr);
    if (rc != HETM_OK) return rc;
    uint32_t gshift = 0;
    while ((4u << gshift) < granule_bytes) ++gshift;
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint32_t blocks = (uint32_t)((n + kSpan - 1) / kSpan);
    // Each launch is checked by its own return code, so that only a failure
    // of this call's launches maps to HETM_ECUDA (an error an unrelated
    // earlier call left pending on this thread is neither reported nor
    // cleared).
    if (blocks) {
        void *args[] = {&dev_log, &n, &dev_rs_bmp, &gshift, &stmr_words, &dev_flag_bits, &scr};
        if (cudaLaunchKernel((const void *)k_validate_noalloc, dim3(blocks), dim3(256), args, 0, s) !=
            cudaSuccess)
            return HETM_ECUDA;
    }
    unsigned long long *count = reinterpret_cast<unsigned long long *>(dev_n_conflicts);
    const NoAllocScratch *cscr = scr;
    void *fargs[] = {&cscr, &blocks, &count, &dev_err};
    if (cudaLaunchKernel((const void *)k_noalloc_finish, dim3(1), dim3(1024), fargs, 0, s) != cudaSuccess)
        return HETM_ECUDA;
    return HETM_OK;
}
