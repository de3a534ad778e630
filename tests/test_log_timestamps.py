"""The CPU log's timestamp rule on the GPU (Sec. IV-C: a tuple is applied when
its timestamp is the newest of its word, and the timestamp totally orders
the writes to one word; needs a GPU).

* Timestamps new to their words in every round: each round leaves the
  oracle's image, the newest timestamp of a word winning.
* A tuple that repeats the timestamp an earlier round applied to its word:
  the round reports HETM_EINVAL, which stays until hetm_load; W and S agree
  on the word and hold its old value or the repeat's, every other word is
  the oracle's.
* Two tuples of one round with the same word and newest timestamp are a
  tie: the round reports HETM_EINVAL, W and S hold one of the two values
  there, every other word is the oracle's.  Ties are placed in the apply's
  full 128-tuple tiles and in its ragged tail.
* A timestamp out of [1, 2^32 - 1) is reported the same way and its tuple is
  not applied; the rest of the log is.

Both conflict policies (the CPU-loses policy raises TS in a pass of its own).
Rounds carry no GPU batch, so they validate clean and apply the whole log.
"""
import numpy as np
import pytest

import oracle
import workloads as wl

pytestmark = pytest.mark.gpu

LOG2W = 14
N = 1 << LOG2W


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def _log(seed, rnd, n, ts_base):
    return wl.cpu_write_log(seed, rnd, n, LOG2W, ts_base=ts_base, cpu_threads=1)[0]


def _state(ctx, h):
    return ctx.read_stmr(h.STMR_W), ctx.read_stmr(h.STMR_S)


@pytest.mark.parametrize("policy", [0, 1])
def test_timestamp_rule(hetm, torch, policy):
    h = hetm
    start = wl.init_words(61, 0, N)
    ts_state = np.zeros(N, dtype=np.uint32)
    cfg = {"cpu_threads": 1, "conflict_policy": policy}
    with h.Context(N, 64, cfg) as ctx:
        ctx.load(start)
        # two rounds of plain logs, the second's timestamps after the first's
        state = start
        applied = {}
        for r in range(2):
            lg = _log(61, r, 1000, 1000 * r)
            ctx.cpu_log_write(0, lg)
            st = ctx.round(stats=True)
            assert st["rc"] == h.HETM_OK and not st["conflict"]
            state, ties = oracle.final_state(state, state, False, lg, ts_state)
            assert ties == 0
            w, s = _state(ctx, h)
            np.testing.assert_array_equal(w, state)
            np.testing.assert_array_equal(s, state)
            for a_, t_ in zip(lg["addr"].tolist(), lg["ts"].tolist()):
                applied[a_] = max(applied.get(a_, 0), t_)

        # new tuples, plus three that repeat, with another value, the
        # timestamp applied to their word earlier
        lg = _log(61, 2, 1000, 2000)
        rep_words = [a_ for a_ in sorted(applied) if a_ not in set(lg["addr"].tolist())][:3]
        rep = np.zeros(3, dtype=wl.LOG_DTYPE)
        rep["addr"] = rep_words
        rep["value"] = [-11, -12, -13]
        rep["ts"] = [applied[a_] for a_ in rep_words]
        lg = np.concatenate([lg[:400], rep, lg[400:]])
        ctx.cpu_log_write(0, lg)
        st = ctx.round(stats=True)
        assert st["rc"] == h.HETM_EINVAL and st["err"] == h.HETM_EINVAL
        prev = state
        state, _ = oracle.final_state(state, state, False, lg, ts_state)
        w, s = _state(ctx, h)
        np.testing.assert_array_equal(w, s)
        for word, v in zip(rep_words, rep["value"].tolist()):
            assert w[word] in (prev[word], v)
        rest = np.ones(N, dtype=bool)
        rest[rep_words] = False
        np.testing.assert_array_equal(w[rest], state[rest])
        # the error stays until hetm_load
        ctx.cpu_log_write(0, _log(61, 3, 100, 5000))
        assert ctx.round(stats=True)["rc"] == h.HETM_EINVAL

        # two ties on words no other tuple of the round names, one pair inside
        # the apply's full 128-tuple tiles, one in its tail
        ctx.load(start)
        ts_state[:] = 0
        lg = _log(61, 4, 1000, 0)
        named = set(lg["addr"].tolist())
        free = [a_ for a_ in range(N) if a_ not in named][:2]
        lg["addr"][[5, 700]] = free[0]
        lg["value"][[5, 700]] = [101, 102]
        lg["ts"][700] = lg["ts"][5]
        lg["addr"][[900, 990]] = free[1]
        lg["value"][[900, 990]] = [201, 202]
        lg["ts"][990] = lg["ts"][900]
        ctx.cpu_log_write(0, lg)
        st = ctx.round(stats=True)
        assert st["rc"] == h.HETM_EINVAL and st["err"] == h.HETM_EINVAL
        expect, ties = oracle.final_state(start, start, False, lg, ts_state)
        assert ties == 2
        w, s = _state(ctx, h)
        for word, pair in zip(free, ((101, 102), (201, 202))):
            assert w[word] in pair and s[word] in pair
        rest = np.ones(N, dtype=bool)
        rest[free] = False
        np.testing.assert_array_equal(w[rest], expect[rest])
        np.testing.assert_array_equal(s[rest], expect[rest])

        # timestamps out of range among valid tuples
        ctx.load(start)
        ts_state[:] = 0
        lg = _log(61, 5, 1000, 0)
        bad = [3, 500, 999]
        lg["ts"][bad] = [0, 0xFFFFFFFF, 0]
        ctx.cpu_log_write(0, lg)
        st = ctx.round(stats=True)
        assert st["rc"] == h.HETM_EINVAL and st["err"] == h.HETM_EINVAL
        keep = np.ones(len(lg), dtype=bool)
        keep[bad] = False
        expect, _ = oracle.final_state(start, start, False, lg[keep], ts_state)
        w, s = _state(ctx, h)
        np.testing.assert_array_equal(w, expect)
        np.testing.assert_array_equal(s, expect)

        # reloaded, a valid log runs clean again
        ctx.load(start)
        ts_state[:] = 0
        lg = _log(61, 6, 1000, 0)
        ctx.cpu_log_write(0, lg)
        assert ctx.round(stats=True)["rc"] == h.HETM_OK
        expect, _ = oracle.final_state(start, start, False, lg, ts_state)
        np.testing.assert_array_equal(ctx.read_stmr(h.STMR_W), expect)
