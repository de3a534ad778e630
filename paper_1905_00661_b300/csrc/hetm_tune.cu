// Autotuner: picks the executor's shape (mode, CTA size, grid, lock table),
// the conflict granule and the WS_bmp / merge chunk for a sample workload by
// running whole synchronization rounds on scratch contexts and timing them.
//
// The paper fixes none of these: its GPU TM runs one kernel shape, and its
// evaluation studies the granule's instrumentation cost against false
// conflicts (Sec. V-A, 4 B vs 1 KB granules) and a 16 KB merge chunk
// (Sec. IV-D).  Here every candidate is measured on the caller's own batches
// and CPU log, with the round's CUDA-event phase times (hetm_round_stats).
//
// Search: three stages of a coordinate search, each starting from the best
// of the one before.
//   stage 0  executor shape: every (mode, exec_threads, blocks per SM,
//            lock_log2) of the space, no CPU log; score = committed per
//            execution-phase second.
//   stage 1  granule: every granule with the CPU log; score = commits of the
//            rounds that validated clean per round second (a conflicting
//            round rolls the GPU batch back), or minus the round time when
//            every candidate conflicts.
//   stage 2  merge chunk: as stage 1.
// A candidate whose warm-up round is slower than `cut` times the best
// warm-up of its stage keeps that one measurement and is not timed further.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "hetm.h"

namespace {

struct Outcome {
    int rc = HETM_OK;
    uint32_t rounds = 0, conflicts = 0;
    uint64_t committed = 0;      // per round (median round)
    uint64_t clean_commits = 0;  // summed over the timed rounds that validated clean
    float ms_exec = 0, ms_round = 0, sum_round = 0;
};

float median(std::vector<float> v) {
    if (v.empty()) return 0;
    std::sort(v.begin(), v.end());
    return v[v.size() / 2];
}

Outcome run_trial(uint64_t words, const int32_t *init, const hetm_batch *b, uint32_t nb,
                  const hetm_log_entry *log, uint64_t n_log, const hetm_config &cfg,
                  uint32_t granule, uint32_t reps, float cut_exec_ms) {
    Outcome o;
    hetm_ctx *c = nullptr;
    o.rc = hetm_init(&c, words, granule, &cfg, nullptr);
    if (o.rc != HETM_OK) return o;
    o.rc = hetm_load(c, init, words);
    std::vector<float> ex, tot;
    std::vector<uint64_t> com;
    for (uint32_t r = 0; o.rc == HETM_OK && r <= reps; ++r) {
        // a timestamp is applied once per word over a context's life, so a
        // round that attaches the same log again starts from a fresh load
        if (r && log && n_log) o.rc = hetm_load(c, init, words);
        for (uint32_t i = 0; o.rc == HETM_OK && i < nb; ++i) o.rc = hetm_gpu_submit_batch(c, b + i, nullptr);
        if (o.rc == HETM_OK && log && n_log) o.rc = hetm_log_attach(c, log, n_log);
        if (o.rc != HETM_OK) break;
        hetm_round_stats st;
        o.rc = hetm_round(c, &st);
        if (o.rc != HETM_OK) break;
        const bool warm = r == 0;
        if (warm && !(cut_exec_ms > 0 && st.ms_exec > cut_exec_ms)) continue;
        ex.push_back(st.ms_exec);
        tot.push_back(st.ms_total);
        com.push_back(st.committed);
        o.sum_round += st.ms_total;
        o.conflicts += st.conflict ? 1u : 0u;
        if (!st.conflict) o.clean_commits += st.committed;
        if (warm) break;  // cut: the warm-up round is its only measurement
    }
    o.rounds = (uint32_t)ex.size();
    o.ms_exec = median(ex);
    o.ms_round = median(tot);
    if (!com.empty()) {
        std::sort(com.begin(), com.end());
        o.committed = com[com.size() / 2];
    }
    hetm_destroy(c);
    return o;
}

float score_exec(const Outcome &o) {
    return o.rc == HETM_OK && o.rounds && o.ms_exec > 0 ? (float)o.committed / (o.ms_exec * 1e-3f) : -1e30f;
}

// commits that survive validation per second of round; rounds that all
// conflict rank by (negative) round time
float score_round(const Outcome &o) {
    if (o.rc != HETM_OK || !o.rounds || o.sum_round <= 0) return -1e30f;
    if (o.clean_commits) return (float)o.clean_commits / (o.sum_round * 1e-3f);
    return -o.ms_round;
}

bool valid_threads(uint32_t mode, uint32_t t) {
    if (mode == HETM_EXEC_ORDERED) return t == 128 || t == 256 || t == 512;
    return t && t % 32 == 0 && t <= 256;
}

}  // namespace

extern "C" {

int hetm_tune_space_default(hetm_tune_space *sp) {
    if (!sp) return HETM_EINVAL;
    std::memset(sp, 0, sizeof(*sp));
    sp->modes = 3;
    sp->threads[0] = 128;
    sp->threads[1] = 256;
    sp->threads[2] = 512;
    sp->blocks_per_sm[0] = 0;  // occupancy limit
    sp->blocks_per_sm[1] = 1;
    sp->lock_log2[0] = 22;
    sp->granules[0] = 4;
    sp->granules[1] = 64;
    sp->granules[2] = 1024;
    sp->ws_chunk_bytes[0] = 1024;
    sp->ws_chunk_bytes[1] = 4096;
    sp->ws_chunk_bytes[2] = 16384;
    sp->reps = 3;
    sp->cut = 4.0f;
    return HETM_OK;
}

int hetm_autotune(uint64_t stmr_words, const int32_t *init, const hetm_batch *batches,
                  uint32_t n_batches, const hetm_log_entry *log, uint64_t n_log,
                  const hetm_config *base, const hetm_tune_space *space, hetm_config *best_cfg,
                  uint32_t *best_granule, hetm_tune_trial *trials, uint32_t max_trials,
                  uint32_t *n_trials) {
    if (!init || !batches || !n_batches || !best_cfg || !best_granule || (n_log && !log) ||
        (max_trials && !trials))
        return HETM_EINVAL;
    hetm_tune_space sp;
    if (space) sp = *space;
    else hetm_tune_space_default(&sp);
    if (!(sp.modes & 3u) || !sp.threads[0] || !sp.granules[0] || !sp.ws_chunk_bytes[0])
        return HETM_EINVAL;
    hetm_config cfg;
    hetm_config_default(&cfg);
    if (base) cfg = *base;
    int n_sm = 0, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return HETM_ECUDA;

    uint32_t n = 0;
    auto record = [&](uint32_t stage, const hetm_config &c, uint32_t g, const Outcome &o, float score) {
        if (n < max_trials) {
            hetm_tune_trial &t = trials[n];
            std::memset(&t, 0, sizeof(t));
            t.stage = stage;
            t.exec_mode = c.exec_mode;
            t.exec_threads = c.exec_threads;
            t.exec_blocks = c.exec_blocks;
            t.lock_log2 = c.lock_log2;
            t.granule_bytes = g;
            t.ws_chunk_bytes = c.ws_chunk_bytes;
            t.rc = o.rc;
            t.rounds = o.rounds;
            t.conflicts = o.conflicts;
            t.committed = o.committed;
            t.ms_exec = o.ms_exec;
            t.ms_round = o.ms_round;
            t.score = score;
        }
        ++n;
    };

    // stage 0: executor shape at the first granule, without the CPU log
    const uint32_t g0 = sp.granules[0];
    hetm_config best = cfg;
    float best_score = -2e30f, best_warm = 0;
    bool any = false;
    for (uint32_t mode = 0; mode < 2; ++mode) {
        if (!(sp.modes & (1u << mode))) continue;
        for (uint32_t ti = 0; ti < 4 && sp.threads[ti]; ++ti) {
            if (!valid_threads(mode, sp.threads[ti])) continue;
            for (uint32_t bi = 0; bi < 4; ++bi) {
                if (bi && !sp.blocks_per_sm[bi]) break;
                const uint32_t nl = mode == HETM_EXEC_OPTIMISTIC ? 4 : 1;
                for (uint32_t li = 0; li < nl; ++li) {
                    if (li && !sp.lock_log2[li]) break;
                    hetm_config c = cfg;
                    c.exec_mode = mode;
                    c.exec_threads = sp.threads[ti];
                    c.exec_blocks = sp.blocks_per_sm[bi] * (uint32_t)n_sm;
                    if (mode == HETM_EXEC_OPTIMISTIC) {
                        if (sp.lock_log2[li]) c.lock_log2 = sp.lock_log2[li];
                        // one lock stripe per cache set region
                        if (c.lock_shift < 4 && cfg.cache_log2_sets) c.lock_shift = 4;
                    }
                    const Outcome o = run_trial(stmr_words, init, batches, n_batches, nullptr, 0, c,
                                                g0, sp.reps, any ? sp.cut * best_warm : 0.f);
                    const float s = score_exec(o);
                    record(0, c, g0, o, s);
                    if (s > best_score) {
                        best_score = s;
                        best = c;
                        best_warm = o.ms_exec;
                        any = true;
                    }
                }
            }
        }
    }
    if (!any) {
        if (n_trials) *n_trials = n;
        return HETM_EINVAL;
    }

    // stage 1: granule, with the CPU log
    uint32_t best_g = g0;
    best_score = -2e30f;
    for (uint32_t gi = 0; gi < 8 && sp.granules[gi]; ++gi) {
        const Outcome o = run_trial(stmr_words, init, batches, n_batches, log, n_log, best,
                                    sp.granules[gi], sp.reps, 0.f);
        const float s = score_round(o);
        record(1, best, sp.granules[gi], o, s);
        if (s > best_score) {
            best_score = s;
            best_g = sp.granules[gi];
        }
    }

    // stage 2: merge chunk
    hetm_config bc = best;
    best_score = -2e30f;
    for (uint32_t ci = 0; ci < 6 && sp.ws_chunk_bytes[ci]; ++ci) {
        hetm_config c = best;
        c.ws_chunk_bytes = sp.ws_chunk_bytes[ci];
        const Outcome o = run_trial(stmr_words, init, batches, n_batches, log, n_log, c, best_g,
                                    sp.reps, 0.f);
        const float s = score_round(o);
        record(2, c, best_g, o, s);
        if (s > best_score) {
            best_score = s;
            bc = c;
        }
    }
    *best_cfg = bc;
    *best_granule = best_g;
    if (n_trials) *n_trials = n;
    return HETM_OK;
}

}  // extern "C"
