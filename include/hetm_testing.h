/*
 * hetm_testing.h -- measurement probes and test scaffolding of the SHeTM
 * round library.  Nothing here is part of a synchronization round: the
 * probes measure the hardware floors that the round's kernels are compared
 * with (their rooflines), and hetm_gpu_mark plants a GPU batch's footprint
 * without running transactions, so that validation and merge can be driven
 * with an exactly known read and write set.
 *
 *   hetm_gpu_mark             -- in libhetm.so (it needs the context)
 *   hetm_handoff_latency,
 *   hetm_random_access_rate,
 *   hetm_l2_probe_rate,
 *   hetm_log_stream_time      -- in libhetm_testing.so
 *
 * Same conventions as hetm.h: 0 = HETM_OK, negative HETM_E* on error.
 */
#ifndef HETM_TESTING_H
#define HETM_TESTING_H

#include "hetm.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Non-transactional instrumentation of words a GPU batch read (vals NULL)
 * or wrote (STMR^W[addr[i]] = vals[i]): the granules go into RS_bmp (and
 * its filter), written words' chunks into WS_bmp, as a committing GPU
 * transaction would record them (Sec. IV-B, IV-C).  addr and vals are
 * device pointers of n entries; an address >= stmr_words is skipped and
 * reported as HETM_EDEVICE by the next call that reads the device error
 * word.  Asynchronous on the context stream. */
HETM_API int hetm_gpu_mark(hetm_ctx *ctx, const uint32_t *addr, const int32_t *vals, uint64_t n);

/* ---------------------------------------------------- handoff latency */
/* Committing in a fixed order serializes the writers of every word, so a
 * batch cannot execute faster than its longest chain of conflicting
 * transactions times the time one transaction needs to hand a word on to
 * the next (the serialization-depth bound).  This measures that hand-on on
 * the current device with nothing else running: *global_ns, a token
 * bounced between two CTAs on two SMs through one global word (acquire
 * load / release store, cooperative launch); *shared_ns, between two warps
 * of one CTA through shared memory.  Each is the mean over 2 x rounds
 * one-way hand-ons.  Either pointer may be NULL.  Synchronous; allocates 40
 * bytes of device memory for the call.  Every wait is bounded (1 s):
 * HETM_ETIMEOUT if one gave up. */
HETM_API int hetm_handoff_latency(uint32_t rounds, double *global_ns, double *shared_ns);

/* Random-sector rate of the current device: n_access random 4-byte reads
 * (*read_per_s) and writes (*write_per_s) spread over a 2^log2_words-word
 * array (20 <= log2_words <= 32; choose it larger than L2 so that every
 * access is a DRAM sector), eight in flight per thread, timed with CUDA
 * events after one warm-up pass.  This is the roofline of scattered work:
 * the executor's word accesses and the apply's timestamp probes and winner
 * writes.  Allocates and frees the array; synchronous.  Either pointer may
 * be NULL, not both. */
HETM_API int hetm_random_access_rate(uint32_t log2_words, uint64_t n_access, double *read_per_s,
                                     double *write_per_s);

/* Random probes of an L2-resident array: n_probe 4-byte loads at hashed
 * positions of a 2^log2_words-word array (10 <= log2_words <= 22; 2^19
 * words = the 2 MiB read-set bitmap of a 2^28-word STMR at 64-byte
 * granules), four independent loads in flight per thread, launched like the
 * validation kernel: one CTA of 1024 threads per SM holding `smem_bytes`
 * (<= 200 KiB) of dynamic shared memory, as the validation kernel's filter
 * does.  *per_s receives probes per second (CUDA events, after one warm-up
 * launch).  This is the probe leg of validation measured alone; the stream
 * leg is the validation kernel on a log none of whose tuples passes the
 * filter.  Allocates and frees the array; synchronous. */
HETM_API int hetm_l2_probe_rate(uint32_t log2_words, uint64_t n_probe, uint32_t smem_bytes,
                                double *per_s);

/* The log stream of validation alone: the address field of each of the n
 * tuples of dev_log (device, 16-byte aligned) read with the validation
 * kernel's loads and launch shape (one 1024-thread CTA per SM holding
 * smem_bytes of shared memory), nothing else done.  *seconds = mean of 10
 * launches after a warm-up (CUDA events), a 256 MiB buffer written before
 * each so that the log does not start in L2.  Allocates 256 MiB for the
 * call; synchronous. */
HETM_API int hetm_log_stream_time(const hetm_log_entry *dev_log, uint64_t n, uint32_t smem_bytes,
                                  double *seconds);

#ifdef __cplusplus
}
#endif
#endif /* HETM_TESTING_H */
