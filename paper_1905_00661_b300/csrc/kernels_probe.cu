// Handoff-latency probe: the floor under one step of a chain of conflicting
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

#include "hetm.h"
#include "hetm_internal.cuh"

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

}  // namespace
}  // namespace hetm

using namespace hetm;

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
