"""Helpers shared by the GPU parity tests: run pieces of a round through the
CUDA library and read back what the oracle is compared with."""
import numpy as np

import workloads as wl


def bits_of(words: np.ndarray) -> np.ndarray:
    """Indices of the set bits of a bitmap of uint32 words (bit g of word g // 32)."""
    b = np.unpackbits(np.ascontiguousarray(words, np.uint32).view(np.uint8), bitorder="little")
    return np.nonzero(b)[0].astype(np.uint32)


def flags_of(words: np.ndarray, n: int) -> np.ndarray:
    b = np.unpackbits(np.ascontiguousarray(words, np.uint32).view(np.uint8), bitorder="little")
    return b[:n].astype(np.uint8)


def to_dev(torch, arr: np.ndarray):
    """Copy a numpy record array to a CUDA byte tensor (16-byte aligned allocation)."""
    raw = np.ascontiguousarray(arr).view(np.uint8).reshape(-1)
    t = torch.empty(max(raw.size, 16), dtype=torch.uint8, device="cuda")
    if raw.size:
        t[: raw.size].copy_(torch.from_numpy(raw))
    return t


class BatchOut:
    """Device output buffers of one batch."""

    def __init__(self, torch, n, out_dtype):
        self.n = n
        self.order = torch.zeros(max(n, 1), dtype=torch.int64, device="cuda")
        self.status = torch.zeros(max(n, 1), dtype=torch.uint8, device="cuda")
        self.out = torch.zeros(max(n, 1), dtype=out_dtype, device="cuda")

    def host(self):
        o = self.order.cpu().numpy().view(np.uint64)[: self.n]
        s = self.status.cpu().numpy()[: self.n]
        r = self.out.cpu().numpy()[: self.n]
        return o, s, r


def submit(ctx, torch, workload, tx, txid_base=0, word_base=0):
    dev = to_dev(torch, tx)
    out_dtype = torch.int64 if workload == wl.WORKLOAD_CACHE else torch.int32
    bo = BatchOut(torch, len(tx), out_dtype)
    ctx.submit_batch(workload, dev, bo.order, bo.status, bo.out, txid_base=txid_base,
                     word_base=word_base, n_tx=len(tx))
    bo.keep = dev
    return bo


def gpu_bitmaps(ctx, h):
    import torch
    torch.cuda.synchronize()
    ctx.sync()
    rs = ctx.device_tensor(h.RS_BMP).cpu().numpy()
    ws = ctx.device_tensor(h.WS_BMP).cpu().numpy()
    return bits_of(rs), bits_of(ws)


def check_keys(order, status):
    """Update commits have distinct even keys; read-only commits odd keys."""
    c = status == 1
    keys = order[c]
    even = keys[keys % 2 == 0]
    assert len(np.unique(even)) == even.size, "two update commits share a version"
    assert (keys > 0).all()
