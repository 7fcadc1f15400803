"""CPU oracle for divide-and-conquer random sampling (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product library shares no code with it.

The C source ``rs_oracle.c`` is the plain, sequential definition of the
sampler (Sec. 3.1 Algorithm R, Sec. 3.2 Algorithm P, Sec. 2 Algorithms H and
B, Sec. 4.6 sampling with replacement, Sec. 4.7 Bernoulli sampling), compiled
with ``-O2 -ffp-contract=off -fno-fast-math`` so that its floating point is
evaluated exactly as written.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rs_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "librs_oracle.so")

CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
          "-fno-strict-aliasing", "-Wall"]

OK, EINVAL, ECAPACITY, ENOMEM, EITER = 0, 1, 2, 3, 6
TAG_SPLIT, TAG_LEAF_H, TAG_LEAF_B, TAG_FIXUP, TAG_BERN, TAG_LEAF_WR = 1, 2, 3, 4, 5, 6
KIND_H, KIND_WR, KIND_B = 0, 1, 2

_lock = threading.Lock()
_lib = None


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"oracle {what} returned {code}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile rs_oracle.c into oracle/_build/librs_oracle.so (if stale)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.run(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        u64, u32, i32, dbl = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_double
        p64 = ctypes.POINTER(ctypes.c_uint64)
        p32 = ctypes.POINTER(ctypes.c_uint32)
        sig = {
            "or_philox4x32_10": (None, [p32, p32, p32]),
            "or_word": (u32, [u64, u32, u64, u64]),
            "or_value": (u64, [u64, u32, u64, u64]),
            "or_u_open": (dbl, [u64]),
            "or_v_closed": (dbl, [u64]),
            "or_candidate": (i32, [u64, u32, u64, u64, u64, p64]),
            "or_log": (dbl, [dbl]),
            "or_log_table_entry": (None, [i32, ctypes.POINTER(dbl), ctypes.POINTER(dbl), ctypes.POINTER(dbl)]),
            "or_log1p": (dbl, [dbl]),
            "or_recip": (dbl, [dbl]),
            "or_log1p_pos": (dbl, [dbl]),
            "or_exp": (dbl, [dbl]),
            "or_lf": (dbl, [u64]),
            "or_lfdiff": (dbl, [u64, u64]),
            "or_sd": (dbl, [u64, u64]),
            "or_sd_fixed": (dbl, [u64, u64, dbl]),
            "or_hg": (i32, [u64, u64, u64, u64, u64, p64]),
            "or_bin": (i32, [u64, u64, u64, u64, u64, p64]),
            "or_depth": (i32, [u64, u64, u32]),
            "or_tree": (i32, [u64, u64, u64, u32, i32, p64, u64, ctypes.POINTER(i32)]),
            "or_leaf_h": (i32, [u64, u64, u64, u64, u64, p64]),
            "or_leaf_wr": (i32, [u64, u64, u64, u64, u64, p64]),
            "or_leaf_b": (i32, [u64, u64, u64, u64, u64, p64]),
            "or_leaf": (i32, [u64, i32, i32, u64, p64, p64]),
            "or_sample": (i32, [u64, u64, u64, u32, i32, p64]),
            "or_range_query": (i32, [u64, u64, u64, u32, i32, u64, u64, p64, u64, p64]),
            "or_bern_chunk_log2": (i32, [dbl, u32]),
            "or_bernoulli": (i32, [dbl, u64, u64, u32, u64, u64, p64, u64, p64]),
            "or_bernoulli_size": (i32, [dbl, u64, u64, p64]),
            "or_union_key": (u64, [u64, u64]),
            "or_points": (i32, [u64, u32, p64, u64, u32, p64]),
            "or_peel_sample": (i32, [u64, u64, u64, u32, p64, p64, u64, p64]),
            "or_union_counts": (i32, [p64, u32, u64, u64, p64]),
            "or_union_sample": (i32, [p64, u32, u64, u64, u32, p64, p64]),
            "or_bernoulli_by_size": (i32, [dbl, u64, u64, u32, u64, u64, p64, u64, p64, p64]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _p64(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def _check(rc: int, what: str):
    if rc != OK:
        raise OracleError(rc, what)


# --- randomness ------------------------------------------------------------

def philox4x32_10(ctr, key):
    """One Philox4x32-10 block for counter (4 words) and key (2 words)."""
    lib = _load()
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (ctypes.c_uint32 * 4)()
    lib.or_philox4x32_10(c, k, o)
    return [int(x) for x in o]


def word(seed, tag, node, j):
    return int(_load().or_word(seed, tag, node, j))


def value(seed, tag, node, j):
    return int(_load().or_value(seed, tag, node, j))


def u_open(x):
    return float(_load().or_u_open(x))


def v_closed(x):
    return float(_load().or_v_closed(x))


def candidate(seed, tag, node, s, j):
    """(valid, value) of candidate j of stream (tag, node) over [0, s)."""
    v = ctypes.c_uint64(0)
    ok = _load().or_candidate(seed, tag, node, s, j, ctypes.byref(v))
    return bool(ok), int(v.value)


# --- math ------------------------------------------------------------------

def log_table_entry(i):
    """Entry i of the logarithm's table: (RN(1/c), hi, lo) with hi + lo = -ln RN(1/c)."""
    inv, hi, lo = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _load().or_log_table_entry(i, ctypes.byref(inv), ctypes.byref(hi), ctypes.byref(lo))
    return inv.value, hi.value, lo.value


def log(x):
    return float(_load().or_log(x))


def log1p(x):
    return float(_load().or_log1p(x))


def recip(x):
    return float(_load().or_recip(x))


def log1p_pos(x):
    return float(_load().or_log1p_pos(x))


def exp(x):
    return float(_load().or_exp(x))


def lf(x):
    return float(_load().or_lf(x))


def lfdiff(x, y):
    return float(_load().or_lfdiff(x, y))


def sd(x, y):
    return float(_load().or_sd(x, y))


def sd_fixed(P, Q, lnP):
    return float(_load().or_sd_fixed(P, Q, lnP))


# --- deviates --------------------------------------------------------------

def hg(seed, node, n, K, S):
    out = ctypes.c_uint64(0)
    _check(_load().or_hg(seed, node, n, K, S, ctypes.byref(out)), "hg")
    return int(out.value)


def binom(seed, node, c, K, S):
    out = ctypes.c_uint64(0)
    _check(_load().or_bin(seed, node, c, K, S, ctypes.byref(out)), "bin")
    return int(out.value)


# --- tree and leaves -------------------------------------------------------

def depth(n, N, n0):
    return int(_load().or_depth(n, N, n0))


def tree(n, N, seed, n0, kind=KIND_H):
    """Leaf records (2^D x 4: lo, s, n', offset) and D."""
    D = depth(n, N, n0)
    L = 1 << D
    recs = np.zeros((L, 4), dtype=np.uint64)
    d = ctypes.c_int(0)
    _check(_load().or_tree(n, N, seed, n0, 1 if kind == KIND_WR else 0, _p64(recs), L, ctypes.byref(d)),
           "tree")
    return recs, D


def leaf(seed, kind, D, i, rec):
    rec = np.ascontiguousarray(rec, dtype=np.uint64)
    out = np.zeros(max(int(rec[2]), 1), dtype=np.uint64)
    _check(_load().or_leaf(seed, kind, D, i, _p64(rec), _p64(out)), "leaf")
    return out[: int(rec[2])]


def leaf_h(seed, node, lo, s, np_):
    out = np.zeros(max(np_, 1), dtype=np.uint64)
    _check(_load().or_leaf_h(seed, node, lo, s, np_, _p64(out)), "leaf_h")
    return out[:np_]


def leaf_wr(seed, node, lo, s, np_):
    out = np.zeros(max(np_, 1), dtype=np.uint64)
    _check(_load().or_leaf_wr(seed, node, lo, s, np_, _p64(out)), "leaf_wr")
    return out[:np_]


def leaf_b(seed, node, lo, s, np_):
    out = np.zeros(max(np_, 1), dtype=np.uint64)
    _check(_load().or_leaf_b(seed, node, lo, s, np_, _p64(out)), "leaf_b")
    return out[:np_]


def sample(n, N, seed, n0=4096, kind=KIND_H):
    """The whole sample: n values from 1..N in non-decreasing order."""
    out = np.zeros(max(n, 1), dtype=np.uint64)
    _check(_load().or_sample(n, N, seed, n0, kind, _p64(out)), "sample")
    return out[:n]


def sample_rc(n, N, seed, n0=4096, kind=KIND_H):
    """Return code of or_sample, for argument checks; n must fit 2^20 slots
    unless the arguments are invalid (then nothing is written)."""
    out = np.zeros(1 << 20, dtype=np.uint64)
    return int(_load().or_sample(n, N, seed, n0, kind, _p64(out)))


def range_query(n, N, seed, n0, kind, a, b, cap=None):
    if cap is None:
        cap = n
    out = np.zeros(max(cap, 1), dtype=np.uint64)
    cnt = ctypes.c_uint64(0)
    rc = _load().or_range_query(n, N, seed, n0, kind, a, b, _p64(out), cap, ctypes.byref(cnt))
    _check(rc, "range_query")
    return out[: int(cnt.value)]


def bern_chunk_log2(p, n0):
    return int(_load().or_bern_chunk_log2(p, n0))


def bernoulli(p, N, seed, n0, a=0, b=None, cap=None):
    """1-based positions of a Bernoulli(p) sample of [0, N) within [a, b)."""
    if b is None:
        b = N
    if cap is None:
        cap = int((b - a) * p + 20 * ((b - a) * p) ** 0.5 + 100)
    out = np.zeros(max(cap, 1), dtype=np.uint64)
    cnt = ctypes.c_uint64(0)
    rc = _load().or_bernoulli(p, N, seed, n0, a, b, _p64(out), cap, ctypes.byref(cnt))
    _check(rc, "bernoulli")
    return out[: int(cnt.value)]


def bernoulli_size(p, N, seed):
    """BIN(N, p) deviate: the size of the Bernoulli sample drawn by its size."""
    cnt = ctypes.c_uint64(0)
    _check(_load().or_bernoulli_size(p, N, seed, ctypes.byref(cnt)), "bernoulli_size")
    return int(cnt.value)


def bernoulli_by_size(p, N, seed, n0, a=0, b=None, cap=None):
    """1-based positions of the Bernoulli(p) sample of [0, N) drawn by its
    size (a BIN(N, p) count, then that many positions without replacement),
    within [a, b); returns (positions, total size)."""
    if b is None:
        b = N
    if cap is None:
        cap = int((b - a) * p + 20 * ((b - a) * p) ** 0.5 + 100)
    out = np.zeros(max(cap, 1), dtype=np.uint64)
    cnt, tot = ctypes.c_uint64(0), ctypes.c_uint64(0)
    rc = _load().or_bernoulli_by_size(p, N, seed, n0, a, b, _p64(out), cap, ctypes.byref(cnt), ctypes.byref(tot))
    _check(rc, "bernoulli_by_size")
    return out[: int(cnt.value)], int(tot.value)


def peel_sample(n, N, seed, n0):
    """(the sample in increasing order, samples per peeled batch)."""
    nb = min(N, 8 * (n // n0 + 1) + 1024) if N else 1
    out = np.zeros(max(n, 1), dtype=np.uint64)
    counts = np.zeros(max(nb, 1), dtype=np.uint64)
    got = ctypes.c_uint64(0)
    _check(_load().or_peel_sample(n, N, seed, n0, _p64(out), _p64(counts), nb, ctypes.byref(got)), "peel_sample")
    return out[:n], counts[: got.value]


def points(n, E, seed, n0):
    """n points uniform in the box [0, E_0) x ... (with replacement), as an
    (n, d) array of 0-based coordinates, leaf after leaf."""
    E = np.ascontiguousarray(E, dtype=np.uint64)
    out = np.zeros(max(n * len(E), 1), dtype=np.uint64)
    _check(_load().or_points(n, len(E), _p64(E), seed, n0, _p64(out)), "points")
    return out[: n * len(E)].reshape(n, len(E))


def union_key(seed, i):
    return int(_load().or_union_key(seed, i))


def union_counts(L, n, seed):
    """Samples per segment of the union sample (binomial tree of HG splits)."""
    L = np.ascontiguousarray(L, dtype=np.uint64)
    counts = np.zeros(max(len(L), 1), dtype=np.uint64)
    _check(_load().or_union_counts(_p64(L), len(L), n, seed, _p64(counts)), "union_counts")
    return counts[: len(L)]


def union_sample(L, n, seed, n0):
    """(positions within their segments, segment after segment; counts)."""
    L = np.ascontiguousarray(L, dtype=np.uint64)
    out = np.zeros(max(n, 1), dtype=np.uint64)
    counts = np.zeros(max(len(L), 1), dtype=np.uint64)
    _check(_load().or_union_sample(_p64(L), len(L), n, seed, n0, _p64(out), _p64(counts)), "union_sample")
    return out[:n], counts[: len(L)]


def bernoulli_rc(p, N, seed, n0, a, b, cap):
    out = np.zeros(max(cap, 1), dtype=np.uint64)
    cnt = ctypes.c_uint64(0)
    rc = _load().or_bernoulli(p, N, seed, n0, a, b, _p64(out), cap, ctypes.byref(cnt))
    return int(rc), int(cnt.value)
