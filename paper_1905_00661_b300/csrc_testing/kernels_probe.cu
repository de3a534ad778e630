// Hardware probes that give the rooflines of the latency- and scatter-bound
// kernels (the memory-copy and GEMM peaks do not describe them).
//
// Handoff latency: the floor under one step of a chain of conflicting
// transactions.  Committing transactions in a fixed order serializes every
// word's writers, so a batch cannot finish faster than its longest chain of
// conflicting transactions times the time one transaction takes to hand a
// word on to the next.  The two kernels here measure that hand-on time with
// nothing else running: a token bounced between two SMs through a global
// word (what a hand-on between CTAs costs), and between two warps of one CTA
// through shared memory (a hand-on inside a CTA segment).
//
// Every wait is bounded (one second of globaltimer); a wait that runs out
// sets *err and both sides return.
#include <cuda_runtime.h>

#include "hetm_internal.cuh"
#include "hetm_testing.h"

namespace hetm {
namespace {

constexpr unsigned long long kProbeLimitNs = 1000000000ull;
constexpr int kProbeSmem = 160 * 1024;  // one CTA per SM: the two CTAs sit on two SMs

__device__ __forceinline__ unsigned long long ld_acq64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_rel64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// CTA b waits for the token to read 2i + b, then writes 2i + b + 1.
__global__ void k_handoff_global(unsigned long long *tok, uint32_t rounds, unsigned long long *out_ns,
                                 int *err) {
    if (threadIdx.x) return;
    const unsigned long long me = blockIdx.x;
    const unsigned long long t0 = globaltimer_ns();
    for (uint32_t i = 0; i < rounds; ++i) {
        const unsigned long long want = 2ull * i + me;
        const unsigned long long ws = globaltimer_ns();
        uint32_t polls = 0;
        while (ld_acq64(tok) != want) {
            if ((++polls & 1023u) == 0) {
                if (*(volatile int *)err) return;
                if (globaltimer_ns() - ws > kProbeLimitNs) {
                    atomicExch(err, 1);
                    return;
                }
            }
        }
        st_rel64(tok, want + 1);
    }
    if (me == 0) out_ns[0] = globaltimer_ns() - t0;
}

// the same between lane 0 of warp 0 and lane 0 of warp 1 of one CTA
__global__ void k_handoff_shared(uint32_t rounds, unsigned long long *out_ns, int *err) {
    __shared__ unsigned long long tok;
    __shared__ int gave_up;
    if (threadIdx.x == 0) {
        tok = 0;
        gave_up = 0;
    }
    __syncthreads();
    if (threadIdx.x & 31u) return;
    volatile unsigned long long *vt = &tok;
    volatile int *vg = &gave_up;
    const unsigned long long me = threadIdx.x >> 5;
    const unsigned long long t0 = globaltimer_ns();
    for (uint32_t i = 0; i < rounds; ++i) {
        const unsigned long long want = 2ull * i + me;
        const unsigned long long ws = globaltimer_ns();
        uint32_t polls = 0;
        while (*vt != want) {
            if ((++polls & 1023u) == 0) {
                if (*vg) return;
                if (globaltimer_ns() - ws > kProbeLimitNs) {
                    *vg = 1;
                    atomicExch(err, 1);
                    return;
                }
            }
        }
        __threadfence_block();
        *vt = want + 1;
    }
    if (me == 0) out_ns[0] = globaltimer_ns() - t0;
}

// Random 4-byte accesses over an array larger than L2: every access touches
// its own 32-byte sector, so accesses/s is the random-sector rate that bounds
// scattered work (the executor's word reads and writes, the apply's TS
// probes and winner writes).  Addresses come from a counter hash; eight
// accesses per thread are in flight at once.
__device__ __forceinline__ uint64_t probe_addr(uint64_t i, uint64_t mask) {
    return splitmix_fin(i * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull) & mask;
}

__global__ void k_gather(const int32_t *__restrict__ x, uint64_t mask, uint64_t n, int32_t *sink) {
    const uint64_t stride = gridDim.x * (uint64_t)blockDim.x;
    int32_t acc = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += 8 * stride) {
        int32_t v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const uint64_t k = i + j * stride;
            v[j] = k < n ? __ldcg(x + probe_addr(k, mask)) : 0;
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) acc ^= v[j];
    }
    if (acc == 0x7FFFFFFF) *sink = acc;  // keeps the loads
}

__global__ void k_scatter(int32_t *x, uint64_t mask, uint64_t n) {
    const uint64_t stride = gridDim.x * (uint64_t)blockDim.x;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += stride)
        x[probe_addr(i, mask)] = (int32_t)i;
}

// Random 4-byte probes of an L2-resident array, four per thread in flight,
// through the same load path (__ldg) as the validation kernel's bitmap probes.
__global__ void __launch_bounds__(1024, 1) k_l2_probe(const uint32_t *__restrict__ x, uint32_t mask,
                                                     uint64_t n, uint32_t *sink) {
    extern __shared__ uint32_t s_hold[];  // occupancy only (the filter's share)
    const uint64_t stride = gridDim.x * (uint64_t)blockDim.x;
    uint32_t acc = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += 4 * stride) {
        uint32_t v[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint64_t k = i + j * stride;
            v[j] = k < n ? __ldg(x + (probe_addr(k, mask) & mask)) : 0u;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) acc ^= v[j];
    }
    if (acc == 0x7FFFFFFFu) {
        s_hold[threadIdx.x] = acc;
        *sink = s_hold[threadIdx.x];  // keeps the loads
    }
}

// The log stream of the validation kernel alone: every tuple's address field
// read with the kernel's loads (4 bytes of every 12, one 32-tuple group per
// warp instruction, 4 groups in flight per warp) and nothing else.
__global__ void __launch_bounds__(1024, 1) k_log_stream(const uint32_t *__restrict__ lw, uint64_t n,
                                                       uint32_t *sink) {
    extern __shared__ uint32_t s_hold2[];  // occupancy only
    constexpr int U = 4;
    const unsigned lane = threadIdx.x & 31u;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t n_warps = (gridDim.x * (uint64_t)blockDim.x) >> 5;
    const uint64_t n_groups = (n + 31) / 32;
    const uint64_t g0 = warp * n_groups / n_warps, g1 = (warp + 1) * n_groups / n_warps;
    uint32_t acc = 0;
    for (uint64_t g = g0; g < g1; g += U) {
        uint32_t a[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint64_t t = (g + u) * 32 + lane;
            uint32_t v = 0;
            if (g + u < g1 && t < n)
                asm volatile("ld.global.nc.L1::no_allocate.u32 %0, [%1];" : "=r"(v) : "l"(lw + 3 * t));
            a[u] = v;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) acc += __ballot_sync(kFull, a[u] & 1u);
    }
    if (acc == 0x12345678u) {
        s_hold2[threadIdx.x] = acc;
        *sink = s_hold2[threadIdx.x];
    }
}

}  // namespace
}  // namespace hetm

using namespace hetm;

extern "C" int hetm_log_stream_time(const hetm_log_entry *dev_log, uint64_t n, uint32_t smem_bytes,
                                    double *seconds) {
    if (!dev_log || n == 0 || smem_bytes > 200u * 1024 || !seconds) return HETM_EINVAL;
    int dev = 0, n_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return HETM_ECUDA;
    uint32_t *sink = nullptr;
    void *flush = nullptr;  // written between launches: more than L2 holds
    const size_t flush_bytes = 256ull << 20;
    if (cudaMalloc(&sink, 64) != cudaSuccess) return HETM_ENOMEM;
    if (cudaMalloc(&flush, flush_bytes) != cudaSuccess) {
        cudaFree(sink);
        return HETM_ENOMEM;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_log_stream, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
    double total = 0;
    const int reps = 10;
    for (int rep = 0; e == cudaSuccess && rep <= reps; ++rep) {  // the first launch warms up
        float ms = 0;
        e = cudaMemsetAsync(flush, rep & 0xFF, flush_bytes);
        if (e == cudaSuccess) e = cudaEventRecord(e0);
        if (e == cudaSuccess) {
            k_log_stream<<<n_sm, 1024, smem_bytes>>>(reinterpret_cast<const uint32_t *>(dev_log), n, sink);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (rep) total += ms * 1e-3;
    }
    if (e == cudaSuccess) *seconds = total / reps;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    cudaFree(flush);
    return e == cudaSuccess ? HETM_OK : HETM_ECUDA;
}

extern "C" int hetm_l2_probe_rate(uint32_t log2_words, uint64_t n_probe, uint32_t smem_bytes,
                                  double *per_s) {
    if (log2_words < 10 || log2_words > 22 || n_probe == 0 || smem_bytes > 200u * 1024 || !per_s)
        return HETM_EINVAL;
    int dev = 0, n_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return HETM_ECUDA;
    const uint64_t words = 1ull << log2_words;
    uint32_t *x = nullptr;
    if (cudaMalloc(&x, words * 4 + 64) != cudaSuccess) return HETM_ENOMEM;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaMemset(x, 0x5A, words * 4 + 64);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_l2_probe, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
    float ms = 0;
    const uint32_t mask = (uint32_t)(words - 1);
    for (int rep = 0; e == cudaSuccess && rep < 3; ++rep) {  // the first launch warms up
        e = cudaEventRecord(e0);
        if (e == cudaSuccess) {
            k_l2_probe<<<n_sm, 1024, smem_bytes>>>(x, mask, n_probe, x + words);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep) {
            const double r = n_probe / (ms * 1e-3);
            if (rep == 1 || r > *per_s) *per_s = r;  // best of two
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(x);
    return e == cudaSuccess ? HETM_OK : HETM_ECUDA;
}

extern "C" int hetm_random_access_rate(uint32_t log2_words, uint64_t n_access, double *read_per_s,
                                       double *write_per_s) {
    if (log2_words < 20 || log2_words > 32 || n_access == 0 || (!read_per_s && !write_per_s))
        return HETM_EINVAL;
    int dev = 0, n_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return HETM_ECUDA;
    const uint64_t words = 1ull << log2_words;
    int32_t *x = nullptr;
    if (cudaMalloc(&x, words * 4 + 64) != cudaSuccess) return HETM_ENOMEM;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaMemset(x, 0, words * 4 + 64);
    const int blocks = n_sm * 8;
    float ms = 0;
    for (int rep = 0; e == cudaSuccess && rep < 2; ++rep) {  // first pass warms up
        if (read_per_s) {
            e = cudaEventRecord(e0);
            k_gather<<<blocks, 256>>>(x, words - 1, n_access, x + words);
            if (e == cudaSuccess) e = cudaEventRecord(e1);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess && rep) *read_per_s = n_access / (ms * 1e-3);
        }
        if (e == cudaSuccess && write_per_s) {
            e = cudaEventRecord(e0);
            k_scatter<<<blocks, 256>>>(x, words - 1, n_access);
            if (e == cudaSuccess) e = cudaEventRecord(e1);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess && rep) *write_per_s = n_access / (ms * 1e-3);
        }
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(x);
    return e == cudaSuccess ? HETM_OK : HETM_ECUDA;
}

extern "C" int hetm_handoff_latency(uint32_t rounds, double *global_ns, double *shared_ns) {
    if (rounds == 0 || rounds > (1u << 24) || (!global_ns && !shared_ns)) return HETM_EINVAL;
    int dev = 0, coop = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess)
        return HETM_ECUDA;
    if (global_ns && !coop) return HETM_EINVAL;
    unsigned long long *buf = nullptr;  // token, two durations
    int *err = nullptr;
    if (cudaMalloc(&buf, 4 * sizeof(unsigned long long)) != cudaSuccess) return HETM_ENOMEM;
    if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) {
        cudaFree(buf);
        return HETM_ENOMEM;
    }
    int rc = HETM_OK;
    unsigned long long h[4] = {0, 0, 0, 0};
    int herr = 0;
    cudaError_t e = cudaMemset(buf, 0, 4 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(err, 0, sizeof(int));
    if (e == cudaSuccess && global_ns) {
        e = cudaFuncSetAttribute(k_handoff_global, cudaFuncAttributeMaxDynamicSharedMemorySize, kProbeSmem);
        unsigned long long *tok = buf, *out = buf + 1;
        void *args[] = {&tok, &rounds, &out, &err};
        // cooperative: both CTAs are resident at once, so neither waits on a
        // CTA that has not started
        if (e == cudaSuccess)
            e = cudaLaunchCooperativeKernel((const void *)k_handoff_global, dim3(2), dim3(32), args,
                                            kProbeSmem, 0);
    }
    if (e == cudaSuccess && shared_ns) {
        k_handoff_shared<<<1, 64>>>(rounds, buf + 2, err);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(h, buf, sizeof(h), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) rc = HETM_ECUDA;
    else if (herr) rc = HETM_ETIMEOUT;
    else {
        if (global_ns) *global_ns = (double)h[1] / (2.0 * rounds);
        if (shared_ns) *shared_ns = (double)h[2] / (2.0 * rounds);
    }
    cudaFree(buf);
    cudaFree(err);
    return rc;
}
