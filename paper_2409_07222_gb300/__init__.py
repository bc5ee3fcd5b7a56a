"""GB300-native hot path of the dual-step LABS search (arXiv 2409.07222).

Thin binding over liblabs.so (include/labs.h): every function here only marshals arguments (torch
tensors for device memory, the current CUDA stream) and calls the C ABI of the same name; all
arithmetic runs in the library's sm_103a kernels.  Packed sequences are int64 (or uint64) tensors of
shape [n, W], W = ceil(L/64): bit (i-1) % 64 of word (i-1) // 64 is 1 iff s_i = +1.
"""
import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import (INT32_MAX, INT32_MIN, LABS_AUTO_THRESHOLD, LABS_MAX_L, LABS_MAX_W, BatchCfg, LabsError,
                   WalkCfg, load, status_string)

CANDIDATE_DTYPE = np.dtype(
    [("E", "<i4"), ("walk", "<u4"), ("step", "<u4"), ("pad", "<u4"), ("fp", "<u8"), ("seq", "<u8", (LABS_MAX_W,))]
)
PQ_STATS_DTYPE = np.dtype(
    [("expansions", "<i8"), ("rounds", "<i8"), ("survivors", "<i8"), ("admitted", "<i8"), ("evicted", "<i8"),
     ("h_size", "<i8"), ("improvements", "<i8"), ("best_fp", "<u8"), ("stop_reason", "<i4"), ("status", "<i4")]
)
WALK_STATS_DTYPE = np.dtype(
    [("flips", "<i8"), ("segments", "<i8"), ("bloom_skips", "<i8"), ("dead_ends", "<i8"), ("E_thr", "<i4"),
     ("best_E", "<i4"), ("status", "<i4"), ("reserved", "<i4")]
)
assert CANDIDATE_DTYPE.itemsize == _lib.CANDIDATE_BYTES and WALK_STATS_DTYPE.itemsize == _lib.WALK_STATS_BYTES
assert PQ_STATS_DTYPE.itemsize == _lib.PQ_STATS_BYTES

_ctxs = {}


def words_per_seq(L):
    return (L + 63) // 64


def context(device=None):
    """The library context of a CUDA device (created on first use)."""
    dev = _device(device)
    idx = dev.index
    if idx not in _ctxs:
        h = ctypes.c_void_p()
        _lib.check(load().labs_ctx_create(ctypes.byref(h), idx), "labs_ctx_create")
        _ctxs[idx] = h
    return _ctxs[idx]


def _device(device):
    if isinstance(device, torch.device):
        return device if device.index is not None else torch.device("cuda", torch.cuda.current_device())
    return torch.device("cuda", torch.cuda.current_device() if device is None else device)


def _stream(device):
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _dev_words(seqs, L):
    if not seqs.is_cuda:
        raise ValueError("sequences must be a CUDA tensor")
    if seqs.dtype not in (torch.int64, torch.uint64):
        raise ValueError("sequences must be int64/uint64 words")
    s = seqs.reshape(-1, words_per_seq(L))
    if not s.is_contiguous():
        s = s.contiguous()
    return s


def labs_energy_batch(seqs, L, with_C=False):
    """E [n] int32 (and C [n, L-1] int32 when with_C) of the packed sequences."""
    s = _dev_words(seqs, L)
    n = s.shape[0]
    E = torch.empty(n, dtype=torch.int32, device=s.device)
    C = torch.empty((n, L - 1), dtype=torch.int32, device=s.device) if with_C else None
    _lib.check(load().labs_energy_batch(context(s.device.index), _ptr(s), L, n, _ptr(E), _ptr(C), _stream(s.device)),
               "labs_energy_batch")
    return (E, C) if with_C else E


def labs_flip_deltas(seqs, L, skew=False, p=0, C=None):
    """dE [n, L] int32: Delta E of every neighbour (position m-1), INT32_MAX outside the free range."""
    s = _dev_words(seqs, L)
    n = s.shape[0]
    dE = torch.empty((n, L), dtype=torch.int32, device=s.device)
    if C is not None:
        C = C.reshape(n, L - 1).to(torch.int32).contiguous()
    _lib.check(load().labs_flip_deltas(context(s.device.index), _ptr(s), _ptr(C), L, n, int(bool(skew)), p, _ptr(dE),
                                       _stream(s.device)), "labs_flip_deltas")
    return dE


def _prefix_tensor(prefixes, p, device):
    pw = max(1, (p + 63) // 64)
    if isinstance(prefixes, torch.Tensor):
        t = prefixes.to(device=device)
        if t.dtype == torch.uint64:
            t = t.view(torch.int64)
    else:
        t = torch.from_numpy(np.ascontiguousarray(np.asarray(prefixes, dtype=np.uint64)).view(np.int64)).to(device)
    return t.reshape(-1, pw).contiguous()


def labs_sample_threshold(L, skew, p, prefixes, seed, n_samples, rank, return_samples=False, device=None):
    """Sieve bound: 0-based `rank`-th smallest energy of n_samples walk-like starts (device int32 [1])."""
    dev = _device(device)
    pre = _prefix_tensor(prefixes, p, dev)
    thr = torch.empty(1, dtype=torch.int32, device=dev)
    samples = torch.empty(n_samples, dtype=torch.int32, device=dev) if return_samples else None
    _lib.check(load().labs_sample_threshold(context(dev.index), L, int(bool(skew)), p, _ptr(pre), pre.shape[0], seed,
                                            n_samples, rank, _ptr(thr), _ptr(samples), _stream(dev)),
               "labs_sample_threshold")
    return (thr, samples) if return_samples else thr


def labs_sample_threshold_noalloc(L, skew, p, prefixes, seed, n_samples, rank, device=None):
    """The sieve bound through the allocation-free entry point (fixed scratch, at most 2^20 samples).

    For callers that may not allocate device memory; ``prefixes`` and the returned int32 [1] tensor
    are the caller's.
    """
    dev = _device(device)
    pre = _prefix_tensor(prefixes, p, dev)
    thr = torch.empty(1, dtype=torch.int32, device=dev)
    with torch.cuda.device(dev):
        _lib.check(load().labs_sample_threshold_noalloc(L, int(bool(skew)), p, _ptr(pre), pre.shape[0], seed,
                                                        n_samples, rank, _ptr(thr), _stream(dev)),
                   "labs_sample_threshold_noalloc")
    return thr


def make_walk_cfg(L, skew=True, p=0, n_walks=1, flip_budget=1000, T_i=0, seed=0, R=16, bloom_log2=15, bloom_k=4,
                  E_thr=INT32_MAX, n_thresh_samples=0, thresh_rank=0, E_target=INT32_MIN, walk_begin=0, tile_m=0,
                  warps_per_cta=0, E_thr_dev=None, lanes_per_walk=0):
    """labs_walk_cfg; E_thr_dev (a device int32 tensor) makes the walk read its sieve bound from it;
    lanes_per_walk 32 / 16 fixes one walk per warp / per half-warp (0: the library chooses)."""
    cfg = WalkCfg()
    cfg.L, cfg.skew, cfg.p, cfg.T_i = L, int(bool(skew)), p, T_i
    cfg.n_walks, cfg.walk_begin, cfg.flip_budget, cfg.seed = n_walks, walk_begin, flip_budget, seed
    cfg.R, cfg.bloom_log2, cfg.bloom_k, cfg.E_thr = R, bloom_log2, bloom_k, E_thr
    cfg.n_thresh_samples, cfg.thresh_rank = n_thresh_samples, thresh_rank
    cfg.E_target, cfg.tile_m, cfg.warps_per_cta = E_target, tile_m, warps_per_cta
    cfg.lanes_per_walk = lanes_per_walk
    cfg.E_thr_dev = E_thr_dev.data_ptr() if E_thr_dev is not None else None
    return cfg


def labs_skew_search(cfg, prefixes, device=None, with_walk_stats=True):
    """Algorithm 1 walks on the device.

    Returns (candidates uint8 [n_walks * R * 96] device tensor, walk_stats int64 [n_walks, 6] or None,
    stats uint8 [48] device tensor).  ``candidates_numpy`` / ``stats_numpy`` decode them.
    """
    dev = _device(device)
    pre = _prefix_tensor(prefixes, cfg.p, dev)
    out = torch.empty(max(1, cfg.n_walks * cfg.R * _lib.CANDIDATE_BYTES), dtype=torch.uint8, device=dev)
    ws = torch.empty((max(1, cfg.n_walks), 6), dtype=torch.int64, device=dev) if with_walk_stats else None
    st = torch.empty(_lib.WALK_STATS_BYTES, dtype=torch.uint8, device=dev)
    _lib.check(load().labs_skew_search(context(dev.index), ctypes.byref(cfg), _ptr(pre), pre.shape[0], _ptr(out),
                                       _ptr(ws), _ptr(st), _stream(dev)), "labs_skew_search")
    return out, ws, st


def make_batch_cfg(n_len, p=24, flip_budget=10000, seed=2410, R=16, bloom_log2=15, bloom_k=4, T_i=0,
                   n_thresh_samples=1000000, thresh_rank=999, E_target=INT32_MIN, tile_m=0, warps_per_cta=0,
                   use_graph=True):
    cfg = BatchCfg()
    cfg.n_len, cfg.p, cfg.flip_budget, cfg.seed = n_len, p, flip_budget, seed
    cfg.R, cfg.bloom_log2, cfg.bloom_k, cfg.T_i = R, bloom_log2, bloom_k, T_i
    cfg.n_thresh_samples, cfg.thresh_rank, cfg.E_target = n_thresh_samples, thresh_rank, E_target
    cfg.tile_m, cfg.warps_per_cta, cfg.use_graph = tile_m, warps_per_cta, int(bool(use_graph))
    return cfg


def labs_batched_search(cfg, lengths, walks, prefixes, device=None, out=None, walk_stats=True):
    """Mixed-length step 1 in one persistent launch (odd lengths skew, even unrestricted).

    Returns (candidates uint8 device tensor [sum(walks) * R * 96], walk_stats int64 [sum(walks), 6] or
    None, per-length sieve bounds int32 [n_len], stats uint8 [48]).  Pass `out` (and reuse the returned
    tensors) to replay the captured graph with the same buffers.
    """
    dev = _device(device)
    Ls = np.ascontiguousarray(np.asarray(lengths, dtype=np.int32))
    Ws = np.ascontiguousarray(np.asarray(walks, dtype=np.int64))
    total = int(Ws.sum())
    pre = _prefix_tensor(prefixes, cfg.p, dev)
    if out is None:
        out = (torch.empty(max(1, total * cfg.R * _lib.CANDIDATE_BYTES), dtype=torch.uint8, device=dev),
               torch.empty((max(1, total), 6), dtype=torch.int64, device=dev) if walk_stats else None,
               torch.empty(len(Ls), dtype=torch.int32, device=dev),
               torch.empty(_lib.WALK_STATS_BYTES, dtype=torch.uint8, device=dev))
    cand, ws, thr, st = out
    _lib.check(load().labs_batched_search(context(dev.index), ctypes.byref(cfg), ctypes.c_void_p(Ls.ctypes.data),
                                          ctypes.c_void_p(Ws.ctypes.data), _ptr(pre), pre.shape[0], _ptr(cand),
                                          _ptr(ws), _ptr(thr), _ptr(st), _stream(dev)), "labs_batched_search")
    return out


def labs_pq_refine(L, seeds, B=4096, cap=1 << 22, H_log2=24, max_expansions=10**7, T_u=0, T_r=0, device=None):
    """Algorithm 2 on the device from packed seed sequences (device int64 [n, W]).

    Returns (best words int64 [W], best E int32 [1], stats uint8 [72]); ``pq_stats_numpy`` decodes stats.
    """
    s = _dev_words(seeds, L)
    dev = s.device
    cfg = _lib.PqCfg()
    cfg.L, cfg.B, cfg.cap, cfg.H_log2, cfg.T_r = L, B, cap, H_log2, T_r
    cfg.max_expansions, cfg.T_u = max_expansions, T_u
    best = torch.empty(words_per_seq(L), dtype=torch.int64, device=dev)
    bE = torch.empty(1, dtype=torch.int32, device=dev)
    st = torch.empty(_lib.PQ_STATS_BYTES, dtype=torch.uint8, device=dev)
    _lib.check(load().labs_pq_refine(context(dev.index), ctypes.byref(cfg), _ptr(s), s.shape[0], _ptr(best), _ptr(bE),
                                     _ptr(st), _stream(dev)), "labs_pq_refine")
    return best, bE, st


def labs_sequence_operators(L, seqs, device=None):
    """The end-element operators: returns (grow int64 [n, 4, W(L+1)], E_grow int32 [n, 4],
    shrink int64 [n, 2, W(L-1)], E_shrink int32 [n, 2]) for packed sequences of length L (device int64)."""
    s = _dev_words(seqs, L)
    dev = s.device
    n = s.shape[0]
    grow = torch.empty((n, 4, words_per_seq(L + 1)), dtype=torch.int64, device=dev)
    Eg = torch.empty((n, 4), dtype=torch.int32, device=dev)
    shrink = torch.empty((n, 2, words_per_seq(L - 1)), dtype=torch.int64, device=dev)
    Es = torch.empty((n, 2), dtype=torch.int32, device=dev)
    _lib.check(load().labs_sequence_operators(context(dev.index), _ptr(s), L, n, _ptr(grow), _ptr(Eg), _ptr(shrink),
                                              _ptr(Es), _stream(dev)), "labs_sequence_operators")
    return grow, Eg, shrink, Es


def labs_seq_to_hex(seq, L):
    """The paper's hexadecimal coding (Section 4) of one packed sequence (host uint64/int64 array [W], or a
    tensor, copied to the host): ceil(L/4) upper-case digits."""
    w = np.ascontiguousarray(seq.cpu().numpy() if torch.is_tensor(seq) else seq).view(np.uint64).reshape(-1)
    if w.size < words_per_seq(L):
        raise ValueError("need %d words for L=%d" % (words_per_seq(L), L))
    buf = ctypes.create_string_buffer((L + 3) // 4 + 1)
    _lib.check(load().labs_seq_to_hex(w.ctypes.data_as(ctypes.c_void_p), L, buf, len(buf)), "labs_seq_to_hex")
    return buf.value.decode()


def labs_hex_to_seq(hex_digits, L):
    """Packed host uint64 [W] of a sequence given in the paper's hexadecimal coding (Section 4)."""
    out = np.zeros(words_per_seq(L), dtype=np.uint64)
    _lib.check(load().labs_hex_to_seq(hex_digits.encode(), L, out.ctypes.data_as(ctypes.c_void_p)), "labs_hex_to_seq")
    return out


ISSUE_RATE_CLASSES = ("IADD", "LOP3", "SHF", "IMAD", "DP4A", "POPC", "PRMT", "FFMA", "DP2A")


def labs_measure_issue_rates(device=None):
    """Measured lane-instructions per SM clock of each class in ISSUE_RATE_CLASSES (dict)."""
    dev = _device(device)
    out = np.zeros(len(ISSUE_RATE_CLASSES), dtype=np.float64)
    _lib.check(load().labs_measure_issue_rates(dev.index, out.ctypes.data_as(ctypes.c_void_p), len(out)),
               "labs_measure_issue_rates")
    return dict(zip(ISSUE_RATE_CLASSES, (float(v) for v in out)))


def labs_legendre_family(L, r_lo=0.20, r_hi=0.24, t_max=0.1):
    """Host enumeration of the Legendre seed family: int32 numpy [n, 2] of (prime p, rotation off)."""
    n = ctypes.c_int64()
    _lib.check(load().labs_legendre_family(L, r_lo, r_hi, t_max, None, 0, ctypes.byref(n)), "labs_legendre_family")
    out = np.zeros((n.value, 2), dtype=np.int32)
    if n.value:
        _lib.check(load().labs_legendre_family(L, r_lo, r_hi, t_max, out.ctypes.data_as(ctypes.c_void_p), n.value,
                                               ctypes.byref(n)), "labs_legendre_family")
    return out


def labs_legendre_construct(L, params, device=None):
    """Seeds for (p, off) pairs (int32 [n, 2], host or device): (packed int64 [n, W], energies int32 [n])."""
    dev = _device(device)
    pr = torch.as_tensor(np.ascontiguousarray(params, dtype=np.int32) if not torch.is_tensor(params) else params,
                         dtype=torch.int32).to(dev).contiguous().reshape(-1, 2)
    n = pr.shape[0]
    seqs = torch.empty((n, words_per_seq(L)), dtype=torch.int64, device=dev)
    E = torch.empty(n, dtype=torch.int32, device=dev)
    _lib.check(load().labs_legendre_construct(context(dev.index), L, _ptr(pr), n, _ptr(seqs), _ptr(E), _stream(dev)),
               "labs_legendre_construct")
    return seqs, E


def labs_pq_independent(L, seeds, max_expansions, T_u=0, T_r=0, H_log2=20, max_workspace_bytes=0, device=None):
    """Algorithm 2 separately for every seed (device int64 [n, W]): (best words [n, W], best E [n], stats [n])."""
    s = _dev_words(seeds, L)
    dev = s.device
    n = s.shape[0]
    cfg = _lib.PqIndepCfg()
    cfg.L, cfg.T_r, cfg.H_log2, cfg.reserved = L, T_r, H_log2, 0
    cfg.max_expansions, cfg.T_u, cfg.max_workspace_bytes = max_expansions, T_u, max_workspace_bytes
    best = torch.empty((n, words_per_seq(L)), dtype=torch.int64, device=dev)
    bE = torch.empty(n, dtype=torch.int32, device=dev)
    st = torch.empty((n, _lib.PQ_STATS_BYTES), dtype=torch.uint8, device=dev)
    _lib.check(load().labs_pq_independent(context(dev.index), ctypes.byref(cfg), _ptr(s), n, _ptr(best), _ptr(bE),
                                          _ptr(st), _stream(dev)), "labs_pq_independent")
    return best, bE, st


def pq_stats_numpy(st):
    return st.cpu().numpy().view(PQ_STATS_DTYPE)[0]


class Policy:
    """The learned flip-proposal network (labs_policy_*): BF16 weights, FP32 accumulation."""

    def __init__(self, L, seed=0, device=None):
        self.dev = _device(device)
        self.L = L
        n = ctypes.c_int64()
        _lib.check(load().labs_policy_param_count(L, ctypes.byref(n)), "labs_policy_param_count")
        self.n_params = n.value
        h = ctypes.c_void_p()
        _lib.check(load().labs_policy_create(context(self.dev.index), L, seed, ctypes.byref(h)), "labs_policy_create")
        self.h = h

    def __del__(self):
        if getattr(self, "h", None) is not None and _lib._lib is not None:
            _lib._lib.labs_policy_destroy(self.h)
            self.h = None

    def set_params(self, flat):
        t = torch.as_tensor(flat, dtype=torch.float32).to(self.dev).contiguous()
        assert t.numel() == self.n_params
        _lib.check(load().labs_policy_set_params(self.h, _ptr(t), _stream(self.dev)), "labs_policy_set_params")
        torch.cuda.current_stream(self.dev).synchronize()

    def get_params(self):
        t = torch.empty(self.n_params, dtype=torch.float32, device=self.dev)
        _lib.check(load().labs_policy_get_params(self.h, _ptr(t), _stream(self.dev)), "labs_policy_get_params")
        return t

    def forward(self, seqs):
        s = _dev_words(seqs, self.L)
        out = torch.empty((s.shape[0], self.L), dtype=torch.float32, device=self.dev)
        _lib.check(load().labs_policy_forward(self.h, _ptr(s), s.shape[0], _ptr(out), _stream(self.dev)),
                   "labs_policy_forward")
        _lib.check(load().labs_policy_sync_status(self.h, _stream(self.dev)), "labs_policy_forward")
        return out

    def train_step(self, seqs, target, weight, free_lo, free_hi, lr, want_grads=False):
        s = _dev_words(seqs, self.L)
        tg = torch.as_tensor(target, dtype=torch.int32).to(self.dev).contiguous()
        wt = torch.as_tensor(weight, dtype=torch.float32).to(self.dev).contiguous()
        loss = torch.empty(1, dtype=torch.float32, device=self.dev)
        grads = torch.empty(self.n_params, dtype=torch.float32, device=self.dev) if want_grads else None
        _lib.check(load().labs_policy_train_step(self.h, _ptr(s), _ptr(tg), _ptr(wt), s.shape[0], free_lo, free_hi,
                                                 float(lr), _ptr(loss), _ptr(grads), _stream(self.dev)),
                   "labs_policy_train_step")
        return loss, grads


def labs_chunked_search(cfg, prefixes, policy=None, lam=0.0, chunk=64, device=None, log_logits=False,
                        log_states=False, log_moves=False, with_walk_stats=True):
    """Algorithm 1 walks in chunks of `chunk` flips, optionally biased by a Policy (learned proposal).

    Returns dict: out, walk_stats, stats (as labs_skew_search) and, when asked, logits [n_chunks, n, L],
    states [n_chunks, n, W] (int64 words), moves [n_chunks, n, 2].
    """
    dev = _device(device)
    pre = _prefix_tensor(prefixes, cfg.p, dev)
    n, L = cfg.n_walks, cfg.L
    nch = (cfg.flip_budget + chunk - 1) // chunk
    res = {
        "out": torch.empty(max(1, n * cfg.R * _lib.CANDIDATE_BYTES), dtype=torch.uint8, device=dev),
        "walk_stats": torch.empty((max(1, n), 6), dtype=torch.int64, device=dev) if with_walk_stats else None,
        "stats": torch.empty(_lib.WALK_STATS_BYTES, dtype=torch.uint8, device=dev),
        "logits": torch.empty((nch, n, L), dtype=torch.float32, device=dev) if log_logits else None,
        "states": torch.empty((nch, n, words_per_seq(L)), dtype=torch.int64, device=dev) if log_states else None,
        "moves": torch.empty((nch, n, 2), dtype=torch.int32, device=dev) if log_moves else None,
    }
    _lib.check(load().labs_chunked_search(context(dev.index), ctypes.byref(cfg), policy.h if policy else None,
                                          float(lam), int(chunk), _ptr(pre), pre.shape[0], _ptr(res["out"]),
                                          _ptr(res["walk_stats"]), _ptr(res["stats"]), _ptr(res["logits"]),
                                          _ptr(res["states"]), _ptr(res["moves"]), _stream(dev)),
               "labs_chunked_search")
    return res


def labs_skew_search_host(cfg, prefixes_host, device=None):
    """End-to-end form: host prefixes in, host candidates/stats out (copies included)."""
    dev = _device(device)
    pre_h = torch.from_numpy(np.ascontiguousarray(np.asarray(prefixes_host, dtype=np.uint64)).view(np.int64))
    pre_h = pre_h.pin_memory()
    pre = pre_h.to(dev, non_blocking=True)
    out, ws, st = labs_skew_search(cfg, pre, device=dev, with_walk_stats=False)
    out_h = torch.empty(out.shape, dtype=torch.uint8, pin_memory=True)
    st_h = torch.empty(st.shape, dtype=torch.uint8, pin_memory=True)
    out_h.copy_(out, non_blocking=True)
    st_h.copy_(st, non_blocking=True)
    torch.cuda.current_stream(dev).synchronize()
    return out_h, st_h


def candidates_numpy(out, n_walks, R):
    a = out.cpu().numpy()[: n_walks * R * _lib.CANDIDATE_BYTES]
    return a.view(CANDIDATE_DTYPE).reshape(n_walks, R)


def stats_numpy(st):
    return st.cpu().numpy().view(WALK_STATS_DTYPE)[0]


def labs_skew_exhaustive(L, p=0, prefix=0, device=None):
    """(min E, count, argmin free-bit integer, argmin packed words) over all skew sequences."""
    dev = _device(device)
    minE = torch.empty(1, dtype=torch.int32, device=dev)
    cnt = torch.empty(1, dtype=torch.int64, device=dev)
    arg = torch.empty(1, dtype=torch.int64, device=dev)
    seq = torch.zeros(words_per_seq(L), dtype=torch.int64, device=dev)
    _lib.check(load().labs_skew_exhaustive(context(dev.index), L, p, prefix, _ptr(minE), _ptr(cnt), _ptr(arg),
                                           _ptr(seq), _stream(dev)), "labs_skew_exhaustive")
    return minE, cnt, arg, seq
