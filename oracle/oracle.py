"""DDQMC oracle binding -- TEST INFRASTRUCTURE ONLY.

Builds ``ddqmc_oracle.c`` with gcc (``-ffp-contract=off`` so that every
floating-point threshold is the same sequence of IEEE operations on any host)
and wraps it with ctypes.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this module.  The product library never
imports it and the oracle never imports the product.

The oracle is a plain single-threaded statement of one step of
driven-dissipative FCIQMC (Nagy & Savona, arXiv:1802.05931, Sec. III.C) with
the initiator rule (Sec. IV.A) and importance sampling (Sec. IV.B).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ddqmc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library in place (seconds)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        u64, i64, i32, dbl = C.c_uint64, C.c_int64, C.c_int32, C.c_double
        P = C.POINTER
        lib.or_create.restype = C.c_void_p
        lib.or_create.argtypes = [C.c_int, C.c_int, C.c_int, dbl, dbl, dbl, dbl, dbl,
                                  i64, i32, C.c_int, dbl, P(dbl), u64, dbl, dbl, i64,
                                  C.c_int, i64, dbl, C.c_int, dbl]
        lib.or_destroy.argtypes = [C.c_void_p]
        lib.or_step.argtypes = [C.c_void_p, i64]
        lib.or_step.restype = C.c_int
        for name in ("or_nobs", "or_nsites", "or_nbonds"):
            getattr(lib, name).argtypes = [C.c_void_p]
            getattr(lib, name).restype = C.c_int
        for name in ("or_size", "or_last_spawns", "or_injected_used"):
            getattr(lib, name).argtypes = [C.c_void_p]
            getattr(lib, name).restype = i64
        lib.or_bonds.argtypes = [C.c_void_p, P(i32), P(i32)]
        lib.or_get_state.argtypes = [C.c_void_p, P(i64), P(dbl), P(i32), P(i64), P(i64), P(i64)]
        lib.or_set_state.argtypes = [C.c_void_p, i64, dbl, i32, i64, i64, i64]
        lib.or_export.argtypes = [C.c_void_p, P(u64), P(u64), P(i32), P(i32), i64]
        lib.or_export.restype = i64
        lib.or_import.argtypes = [C.c_void_p, P(u64), P(u64), P(i32), P(i32), i64]
        lib.or_import.restype = C.c_int
        lib.or_estimates_now.argtypes = [C.c_void_p, P(i64)]
        lib.or_series.argtypes = [C.c_void_p, P(i64), i64]
        lib.or_series.restype = i64
        lib.or_moves.argtypes = [C.c_void_p, u64, u64, P(u64), P(u64), P(i32), P(dbl), P(dbl), P(u64)]
        lib.or_moves.restype = C.c_int
        lib.or_diag.argtypes = [C.c_void_p, u64, u64, P(dbl), P(dbl)]
        lib.or_inject.argtypes = [C.c_void_p, P(C.c_uint32), i64]
        lib.or_inject.restype = C.c_int
        lib.or_philox4x32_10.argtypes = [P(C.c_uint32), P(C.c_uint32), P(C.c_uint32)]
        lib.or_annihilate.argtypes = [P(u64), P(u64), P(i32), P(i32), i64, P(u64), P(u64), P(i32), P(i32),
                                      P(i32), i64, i32, P(u64), P(u64), P(i32), P(i32), i64]
        lib.or_annihilate.restype = i64
        lib.or_gather.argtypes = [C.c_void_p, P(u64), P(u64), P(i32), P(i32), i64, P(u64), P(u64), i64,
                                  P(i64), P(i64)]
        lib.or_gather.restype = C.c_int
        lib.or_series_log.argtypes = [dbl]
        lib.or_series_log.restype = dbl
        _lib = lib
        return lib


def _ptr(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def philox4x32_10(ctr, key):
    """Philox4x32-10 of one counter block (Salmon et al., SC'11)."""
    lib = _load()
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib.or_philox4x32_10(_ptr(c, C.c_uint32), _ptr(k, C.c_uint32), _ptr(out, C.c_uint32))
    return [int(x) for x in out]


def annihilate(lket, lbra, lre, lim, sket, sbra, sre, sim, sinit, n_a):
    """Annihilation of a sorted list with unsorted spawn records under the
    initiator rule (Sec. III.C rule (iii), Sec. IV.A); returns the merged list."""
    lib = _load()
    a = [np.ascontiguousarray(x, dtype=t) for x, t in ((lket, np.uint64), (lbra, np.uint64), (lre, np.int32),
                                                     (lim, np.int32))]
    b = [np.ascontiguousarray(x, dtype=t) for x, t in ((sket, np.uint64), (sbra, np.uint64), (sre, np.int32),
                                                     (sim, np.int32), (sinit, np.int32))]
    cap = len(a[0]) + len(b[0])
    o = [np.zeros(max(cap, 1), dtype=t) for t in (np.uint64, np.uint64, np.int32, np.int32)]
    cts = (C.c_uint64, C.c_uint64, C.c_int32, C.c_int32)
    n = lib.or_annihilate(*[_ptr(x, ct) for x, ct in zip(a, cts)], len(a[0]),
                          *[_ptr(x, ct) for x, ct in zip(b, cts + (C.c_int32,))], len(b[0]), int(n_a),
                          *[_ptr(x, ct) for x, ct in zip(o, cts)], cap)
    if n < 0:
        raise RuntimeError("oracle annihilation failed (%d)" % n)
    return tuple(x[:n] for x in o)


def series_log(x: float) -> float:
    """The deterministic series logarithm used by the shift update."""
    return _load().or_series_log(float(x))


class OracleRun:
    """One DDQMC run on the CPU.  Parameters mirror the C-ABI ``ddqmc_create``;
    field_axis = 2 takes the field angle field_theta."""

    def __init__(self, Lx, Ly, periodic, Jx, Jy, Jz, gamma, dt, target, n_a=0,
                 guide_kind=0, guide_p=0.0, site_ratio=None, seed=1, damping=0.05,
                 shift0=-1.0, n0=1000, control=0, t_eq=-1, field_h=0.0, field_axis=0, field_theta=0.0):
        lib = _load()
        self._lib = lib
        self._site_r = None
        rp = None
        if site_ratio is not None:
            self._site_r = np.ascontiguousarray(site_ratio, dtype=np.float64)
            rp = _ptr(self._site_r, C.c_double)
        h = lib.or_create(int(Lx), int(Ly), int(periodic), float(Jx), float(Jy), float(Jz),
                          float(gamma), float(dt), int(target), int(n_a), int(guide_kind),
                          float(guide_p), rp, int(seed) & ((1 << 64) - 1), float(damping),
                          float(shift0), int(n0), int(control), int(t_eq), float(field_h), int(field_axis),
                          float(field_theta))
        if not h:
            raise ValueError("oracle rejected the parameters")
        self._h = C.c_void_p(h)
        self.N = lib.or_nsites(self._h)
        self.B = lib.or_nbonds(self._h)
        self.nobs = lib.or_nobs(self._h)
        self.n_a = int(n_a)
        self.field_h = float(field_h)
        self._inj = None

    def close(self):
        if getattr(self, "_h", None):
            self._lib.or_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- stepping -----------------------------------------------------------
    def step(self, n=1):
        rc = self._lib.or_step(self._h, int(n))
        if rc != 0:
            raise RuntimeError("oracle step failed with code %d" % rc)

    def inject(self, uniforms):
        """Use the given 32-bit words instead of Philox (None restores Philox).
        Returns True if the previous injected stream ran short."""
        if uniforms is None:
            self._inj = None
            return bool(self._lib.or_inject(self._h, None, 0))
        self._inj = np.ascontiguousarray(uniforms, dtype=np.uint32)
        return bool(self._lib.or_inject(self._h, _ptr(self._inj, C.c_uint32), len(self._inj)))

    def injected_used(self):
        return int(self._lib.or_injected_used(self._h))

    # --- state --------------------------------------------------------------
    def bonds(self):
        a = np.zeros(self.B, dtype=np.int32)
        b = np.zeros(self.B, dtype=np.int32)
        self._lib.or_bonds(self._h, _ptr(a, C.c_int32), _ptr(b, C.c_int32))
        return list(zip(a.tolist(), b.tolist()))

    def state(self):
        t, S, var, Q, tv, te = C.c_int64(), C.c_double(), C.c_int32(), C.c_int64(), C.c_int64(), C.c_int64()
        self._lib.or_get_state(self._h, C.byref(t), C.byref(S), C.byref(var), C.byref(Q),
                               C.byref(tv), C.byref(te))
        return dict(t=t.value, S=S.value, variable=var.value, Qprev=Q.value,
                    t_var=tv.value, t_eq=te.value)

    def set_state(self, t, S, variable, Qprev, t_var, t_eq):
        self._lib.or_set_state(self._h, int(t), float(S), int(variable), int(Qprev),
                               int(t_var), int(t_eq))

    def size(self):
        return int(self._lib.or_size(self._h))

    def last_spawns(self):
        return int(self._lib.or_last_spawns(self._h))

    def export(self):
        n = self.size()
        ket = np.zeros(n, dtype=np.uint64)
        bra = np.zeros(n, dtype=np.uint64)
        re = np.zeros(n, dtype=np.int32)
        im = np.zeros(n, dtype=np.int32)
        self._lib.or_export(self._h, _ptr(ket, C.c_uint64), _ptr(bra, C.c_uint64),
                            _ptr(re, C.c_int32), _ptr(im, C.c_int32), n)
        return ket, bra, re, im

    def import_(self, ket, bra, re, im):
        ket = np.ascontiguousarray(ket, dtype=np.uint64)
        bra = np.ascontiguousarray(bra, dtype=np.uint64)
        re = np.ascontiguousarray(re, dtype=np.int32)
        im = np.ascontiguousarray(im, dtype=np.int32)
        rc = self._lib.or_import(self._h, _ptr(ket, C.c_uint64), _ptr(bra, C.c_uint64),
                                 _ptr(re, C.c_int32), _ptr(im, C.c_int32), len(ket))
        if rc != 0:
            raise ValueError("oracle import rejected the list (code %d)" % rc)

    def estimates_now(self):
        out = np.zeros(self.nobs, dtype=np.int64)
        self._lib.or_estimates_now(self._h, _ptr(out, C.c_int64))
        return out

    def series(self):
        n = int(self._lib.or_series(self._h, None, 0))
        out = np.zeros((max(n, 1), self.nobs), dtype=np.int64)
        self._lib.or_series(self._h, _ptr(out, C.c_int64), n)
        return out[:n]

    def gather(self, ket, bra, re, im, tket, tbra):
        """One step of the list (ket, bra, re, im) -- sorted by (bra, ket),
        unique -- evaluated only at the targets (tket, tbra), at this run's t
        and S: the targets' entries of the stepped list, (0, 0) where a target
        is absent from it.  The run's own list is not touched."""
        a = [np.ascontiguousarray(x, dtype=t) for x, t in ((ket, np.uint64), (bra, np.uint64), (re, np.int32),
                                                         (im, np.int32))]
        tk = np.ascontiguousarray(tket, dtype=np.uint64)
        tb = np.ascontiguousarray(tbra, dtype=np.uint64)
        ore = np.zeros(len(tk), dtype=np.int64)
        oim = np.zeros(len(tk), dtype=np.int64)
        rc = self._lib.or_gather(self._h, _ptr(a[0], C.c_uint64), _ptr(a[1], C.c_uint64), _ptr(a[2], C.c_int32),
                                 _ptr(a[3], C.c_int32), len(a[0]), _ptr(tk, C.c_uint64), _ptr(tb, C.c_uint64),
                                 len(tk), _ptr(ore, C.c_int64), _ptr(oim, C.c_int64))
        if rc != 0:
            raise RuntimeError("oracle gather failed with code %d" % rc)
        return ore, oim

    # --- element access for the Liouvillian pins ----------------------------
    def moves(self, i, j):
        K = 2 * self.B + 5 * self.N
        ck = np.zeros(K, dtype=np.uint64)
        cb = np.zeros(K, dtype=np.uint64)
        kind = np.zeros(K, dtype=np.int32)
        are = np.zeros(K, dtype=np.float64)
        aim = np.zeros(K, dtype=np.float64)
        rate = np.zeros(K, dtype=np.uint64)
        n = self._lib.or_moves(self._h, int(i), int(j), _ptr(ck, C.c_uint64), _ptr(cb, C.c_uint64),
                               _ptr(kind, C.c_int32), _ptr(are, C.c_double), _ptr(aim, C.c_double),
                               _ptr(rate, C.c_uint64))
        return ck[:n], cb[:n], kind[:n], are[:n] + 1j * aim[:n], rate[:n]

    def diag(self, i, j):
        dr, di = C.c_double(), C.c_double()
        self._lib.or_diag(self._h, int(i), int(j), C.byref(dr), C.byref(di))
        return complex(dr.value, di.value)


def observable_layout(N, B):
    """Index map of the integer estimator vector (same layout on both sides)."""
    oz = 5
    ozz = oz + N
    oxx = ozz + B
    oyy = oxx + B
    oag = oyy + B
    ox = oag + 4
    oy = ox + N
    return dict(tr=0, tr_im=1, nw=2, walkers=3, entries=4, z=oz, zz=ozz, xx=oxx, yy=oyy,
                sum_z=oag, sum_zz=oag + 1, sum_xx=oag + 2, sum_yy=oag + 3, x=ox, y=oy,
                sum_x=oy + N, sum_y=oy + N + 1, nobs=oy + N + 2)
