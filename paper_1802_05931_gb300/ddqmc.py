"""Python binding of libddqmc.so (argument marshalling only).

Every function here has the name of the C entry point it calls (see
include/ddqmc.h); every step of the DDQMC path runs in the library's CUDA
kernels.  The binding raises if the library has not been built: there is no
CPU fallback.  ``Run`` is a small convenience wrapper over the same calls.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libddqmc.so")

MAX_SITES = 64
MAX_BONDS = 128
MAX_BATCH = 64

ERRORS = {0: "OK", -1: "INVALID_ARG", -2: "OOM", -3: "CAPACITY", -4: "OVERFLOW", -5: "TIMEOUT",
          -6: "CUDA", -7: "UNSUPPORTED"}


class DDQMCError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__("%s failed: %s (%d)" % (what, ERRORS.get(code, "?"), code))


class ddqmc_tuning(C.Structure):
    _fields_ = [("spawn_blocks_per_sm", C.c_int32), ("radix_blocks_per_sm", C.c_int32),
                ("merge_blocks_per_sm", C.c_int32), ("copy_blocks_per_sm", C.c_int32),
                ("scan_blocks_per_sm", C.c_int32), ("partition_blocks_per_sm", C.c_int32),
                ("heavy_walkers", C.c_int32), ("radix_records_per_thread", C.c_int32),
                ("step_ms_default", C.c_double), ("step_ms_tuned", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ddqmc_lattice(C.Structure):
    _fields_ = [("Lx", C.c_int32), ("Ly", C.c_int32), ("periodic", C.c_int32)]


class ddqmc_guide(C.Structure):
    _fields_ = [("kind", C.c_int32), ("p", C.c_double), ("site_ratio", C.POINTER(C.c_double))]


class ddqmc_options(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("damping", C.c_double), ("shift0", C.c_double),
                ("n0", C.c_int64), ("control", C.c_int32), ("t_eq", C.c_int64),
                ("capacity_entries", C.c_int64), ("capacity_spawns", C.c_int64),
                ("cuda_stream", C.c_void_p), ("sm_limit", C.c_int32), ("field_h", C.c_double),
                ("field_axis", C.c_int32), ("wide_sort_bits", C.c_int32), ("field_theta", C.c_double)]


class ddqmc_estimates(C.Structure):
    _fields_ = [("t", C.c_int64), ("shift", C.c_double), ("variable", C.c_int32),
                ("t_var", C.c_int64), ("t_eq", C.c_int64), ("n_samples", C.c_int64),
                ("walkers", C.c_int64), ("entries", C.c_int64), ("nw", C.c_int64),
                ("trace_re", C.c_int64), ("trace_im", C.c_int64),
                ("nsites", C.c_int32), ("nbonds", C.c_int32), ("walker_steps", C.c_double),
                ("mz", C.c_double), ("mz_err", C.c_double),
                ("xx", C.c_double), ("xx_err", C.c_double), ("yy", C.c_double), ("yy_err", C.c_double),
                ("zz", C.c_double), ("zz_err", C.c_double),
                ("sz", C.c_double * MAX_SITES), ("sz_err", C.c_double * MAX_SITES),
                ("bond_xx", C.c_double * MAX_BONDS), ("bond_yy", C.c_double * MAX_BONDS),
                ("bond_zz", C.c_double * MAX_BONDS),
                ("mx", C.c_double), ("mx_err", C.c_double), ("my", C.c_double), ("my_err", C.c_double),
                ("sx", C.c_double * MAX_SITES), ("sy", C.c_double * MAX_SITES)]


class ddqmc_run_spec(C.Structure):
    _fields_ = [("Jx", C.c_double), ("Jy", C.c_double), ("Jz", C.c_double), ("gamma", C.c_double),
                ("dt", C.c_double), ("target_walkers", C.c_int64), ("initiator_threshold", C.c_int32),
                ("control", C.c_int32), ("seed", C.c_uint64), ("damping", C.c_double), ("shift0", C.c_double),
                ("n0", C.c_int64), ("t_eq", C.c_int64), ("field_h", C.c_double), ("field_axis", C.c_int32),
                ("reserved", C.c_int32), ("field_theta", C.c_double)]


class ddqmc_state(C.Structure):
    _fields_ = [("t", C.c_int64), ("shift", C.c_double), ("variable", C.c_int32),
                ("q_prev", C.c_int64), ("t_var", C.c_int64), ("t_eq", C.c_int64),
                ("entries", C.c_int64), ("status", C.c_int32), ("status_bits", C.c_int32)]


EXPORTS = ["ddqmc_default_options", "ddqmc_create", "ddqmc_step", "ddqmc_step_async", "ddqmc_sync",
           "ddqmc_estimators", "ddqmc_raw_estimators", "ddqmc_blocking_moments",
           "ddqmc_export_walkers", "ddqmc_import_walkers", "ddqmc_export_records", "ddqmc_import_records",
           "ddqmc_export_records32", "ddqmc_import_records32",
           "ddqmc_get_state", "ddqmc_get_counts",
           "ddqmc_get_totals", "ddqmc_set_timing", "ddqmc_get_timing", "ddqmc_tune", "ddqmc_set_tuning",
           "ddqmc_get_tuning", "ddqmc_annihilate",
           "ddqmc_annihilate_noalloc", "ddqmc_wait_selftest", "ddqmc_create_batch", "ddqmc_batch_estimators",
           "ddqmc_batch_raw_estimators", "ddqmc_batch_export_walkers", "ddqmc_batch_get_state", "ddqmc_batch_retire",
           "ddqmc_destroy",
           "ddqmc_strerror"]
NOALLOC_MAX_SPAWNS = 1 << 18
NOALLOC_MAX_LIST = 1 << 20
KERNEL_CLASSES = ["spawn_death", "radix_pass", "merge_partition", "merge", "finalize", "merge_compact"]

_lib = None


def load(path: str = LIB_PATH):
    """Load libddqmc.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libddqmc.so is not built (run __graft_entry__.build()); "
                           "the DDQMC path has no CPU fallback")
    lib = C.CDLL(path)
    P = C.POINTER
    i32, i64, u64, dbl, vp = C.c_int32, C.c_int64, C.c_uint64, C.c_double, C.c_void_p
    lib.ddqmc_default_options.argtypes = [P(ddqmc_options)]
    lib.ddqmc_create.argtypes = [P(ddqmc_lattice), dbl, dbl, dbl, dbl, dbl, i64, i32, P(ddqmc_guide),
                                 P(ddqmc_options), P(vp)]
    lib.ddqmc_step.argtypes = [vp, i64]
    lib.ddqmc_step_async.argtypes = [vp, i64]
    lib.ddqmc_sync.argtypes = [vp]
    lib.ddqmc_estimators.argtypes = [vp, P(ddqmc_estimates)]
    lib.ddqmc_raw_estimators.argtypes = [vp, P(i64), i32, P(i32)]
    lib.ddqmc_blocking_moments.argtypes = [vp, i32, i32, P(i64), P(i64), P(i64), P(i64)]
    lib.ddqmc_export_walkers.argtypes = [vp, P(u64), P(u64), P(i32), P(i32), i64, P(i64)]
    lib.ddqmc_export_records.argtypes = [vp, vp, i64, P(i64)]
    lib.ddqmc_import_records.argtypes = [vp, vp, i64, i64, dbl, i32, i64, i64, i64]
    lib.ddqmc_export_records32.argtypes = [vp, vp, i64, P(i64)]
    lib.ddqmc_import_records32.argtypes = [vp, vp, i64, i64, dbl, i32, i64, i64, i64]
    lib.ddqmc_import_walkers.argtypes = [vp, P(u64), P(u64), P(i32), P(i32), i64, i64, dbl, i32, i64,
                                         i64, i64]
    lib.ddqmc_get_state.argtypes = [vp, P(ddqmc_state)]
    lib.ddqmc_get_counts.argtypes = [vp, P(i64), P(i64), P(i64)]
    lib.ddqmc_get_totals.argtypes = [vp, P(i64), P(i64), P(i64), P(i64)]
    lib.ddqmc_set_timing.argtypes = [vp, i32]
    lib.ddqmc_get_timing.argtypes = [vp, P(dbl), P(i64), i32]
    lib.ddqmc_annihilate.argtypes = [vp, vp, i64, vp, i64, vp, i64, P(i64)]
    lib.ddqmc_annihilate_noalloc.argtypes = [P(ddqmc_lattice), i32, vp, i64, vp, i64, vp, i64, P(i64), vp]
    lib.ddqmc_wait_selftest.argtypes = [vp]
    lib.ddqmc_create_batch.argtypes = [P(ddqmc_lattice), i32, P(ddqmc_run_spec), P(ddqmc_guide), P(ddqmc_options),
                                       P(vp)]
    lib.ddqmc_batch_estimators.argtypes = [vp, i32, P(ddqmc_estimates)]
    lib.ddqmc_batch_raw_estimators.argtypes = [vp, i32, P(i64), i32, P(i32)]
    lib.ddqmc_batch_export_walkers.argtypes = [vp, i32, P(u64), P(u64), P(i32), P(i32), i64, P(i64)]
    lib.ddqmc_batch_get_state.argtypes = [vp, i32, P(ddqmc_state)]
    lib.ddqmc_batch_retire.argtypes = [vp, i32]
    lib.ddqmc_tune.argtypes = [vp, P(ddqmc_tuning)]
    lib.ddqmc_set_tuning.argtypes = [vp, P(ddqmc_tuning)]
    lib.ddqmc_get_tuning.argtypes = [vp, P(ddqmc_tuning)]
    lib.ddqmc_destroy.argtypes = [vp]
    lib.ddqmc_destroy.restype = None
    lib.ddqmc_strerror.argtypes = [C.c_int]
    lib.ddqmc_strerror.restype = C.c_char_p
    for n in EXPORTS:
        if n not in ("ddqmc_destroy", "ddqmc_strerror"):
            getattr(lib, n).restype = C.c_int
    _lib = lib
    return lib


def _check(rc, what):
    if rc != 0:
        raise DDQMCError(rc, what)


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


# --- thin wrappers with the C names -------------------------------------------------------
def ddqmc_default_options():
    o = ddqmc_options()
    _check(load().ddqmc_default_options(C.byref(o)), "ddqmc_default_options")
    return o


def ddqmc_create(lattice, Jx, Jy, Jz, gamma, dt, target_walkers, initiator_threshold, guide=None,
                 options=None):
    lib = load()
    h = C.c_void_p()
    rc = lib.ddqmc_create(C.byref(lattice), Jx, Jy, Jz, gamma, dt, int(target_walkers),
                          int(initiator_threshold), C.byref(guide) if guide is not None else None,
                          C.byref(options) if options is not None else None, C.byref(h))
    _check(rc, "ddqmc_create")
    return h


def ddqmc_step(run, nsteps):
    return load().ddqmc_step(run, int(nsteps))


def ddqmc_step_async(run, nsteps):
    return load().ddqmc_step_async(run, int(nsteps))


def ddqmc_sync(run):
    return load().ddqmc_sync(run)


def ddqmc_estimators(run):
    e = ddqmc_estimates()
    rc = load().ddqmc_estimators(run, C.byref(e))
    return rc, e


def ddqmc_raw_estimators(run, cap=1024):
    out = np.zeros(cap, dtype=np.int64)
    n = C.c_int32()
    _check(load().ddqmc_raw_estimators(run, _p(out, C.c_int64), cap, C.byref(n)), "ddqmc_raw_estimators")
    return out[: n.value]


def ddqmc_blocking_moments(run, k, levels=32):
    n = np.zeros(levels, dtype=np.int64)
    sx = np.zeros(levels, dtype=np.int64)
    sxx = np.zeros(2 * levels, dtype=np.int64)
    sxy = np.zeros(2 * levels, dtype=np.int64)
    _check(load().ddqmc_blocking_moments(run, int(k), levels, _p(n, C.c_int64), _p(sx, C.c_int64),
                                         _p(sxx, C.c_int64), _p(sxy, C.c_int64)), "ddqmc_blocking_moments")

    def i128(a, l):
        return (int(a[2 * l + 1]) << 64) + (int(a[2 * l]) & ((1 << 64) - 1))
    return [dict(n=int(n[l]), sx=int(sx[l]), sxx=i128(sxx, l), sxy=i128(sxy, l)) for l in range(levels)]


def ddqmc_export_walkers(run, out=None):
    """(ket, bra, re, im) of the current list; `out` may hold four arrays of
    those dtypes to write into (reused when long enough, e.g. between steps)."""
    lib = load()
    return _export(lambda *a: lib.ddqmc_export_walkers(run, *a), out, "ddqmc_export_walkers")


# the run's own 16-byte list records (ddqmc_export_records / ddqmc_import_records)
RECORD_DTYPE = np.dtype([("key", "<u8"), ("re", "<i4"), ("im", "<i4")])
# 12-byte records of keys of at most 32 bits (ddqmc_export_records32 / ddqmc_import_records32)
RECORD32_DTYPE = np.dtype([("key", "<u4"), ("re", "<i4"), ("im", "<i4")])


def ddqmc_export_records(run, out=None):
    """The current list as RECORD_DTYPE records (key = bra << N | ket); `out`
    (a RECORD_DTYPE array, e.g. pinned) is written into when long enough."""
    lib = load()
    n = C.c_int64()
    _check(lib.ddqmc_export_records(run, None, 0, C.byref(n)), "ddqmc_export_records")
    m = n.value
    if out is None or len(out) < m or out.dtype != RECORD_DTYPE or not out.flags.c_contiguous:
        out = np.empty(max(m, 1), dtype=RECORD_DTYPE)
    _check(lib.ddqmc_export_records(run, out.ctypes.data_as(C.c_void_p), len(out), C.byref(n)),
           "ddqmc_export_records")
    return out[:m]


def ddqmc_import_records(run, recs, t, S, variable=0, q_prev=1, t_var=-1, t_eq=-1):
    recs = np.ascontiguousarray(recs, dtype=RECORD_DTYPE)
    _check(load().ddqmc_import_records(run, recs.ctypes.data_as(C.c_void_p), len(recs), int(t), float(S),
                                       int(variable), int(q_prev), int(t_var), int(t_eq)), "ddqmc_import_records")


def ddqmc_export_records32(run, out=None):
    """The current list as RECORD32_DTYPE records (lattices of at most 16 sites)."""
    lib = load()
    n = C.c_int64()
    _check(lib.ddqmc_export_records32(run, None, 0, C.byref(n)), "ddqmc_export_records32")
    m = n.value
    if out is None or len(out) < m or out.dtype != RECORD32_DTYPE or not out.flags.c_contiguous:
        out = np.empty(max(m, 1), dtype=RECORD32_DTYPE)
    _check(lib.ddqmc_export_records32(run, out.ctypes.data_as(C.c_void_p), len(out), C.byref(n)),
           "ddqmc_export_records32")
    return out[:m]


def ddqmc_import_records32(run, recs, t, S, variable=0, q_prev=1, t_var=-1, t_eq=-1):
    recs = np.ascontiguousarray(recs, dtype=RECORD32_DTYPE)
    _check(load().ddqmc_import_records32(run, recs.ctypes.data_as(C.c_void_p), len(recs), int(t), float(S),
                                         int(variable), int(q_prev), int(t_var), int(t_eq)),
           "ddqmc_import_records32")


def ddqmc_batch_export_walkers(batch, k, out=None):
    """(ket, bra, re, im) of run k of a batch (as ddqmc_export_walkers)."""
    lib = load()
    return _export(lambda *a: lib.ddqmc_batch_export_walkers(batch, int(k), *a), out, "ddqmc_batch_export_walkers")


def _export(call, out, what):
    n = C.c_int64()
    _check(call(None, None, None, None, 0, C.byref(n)), what)
    m = n.value
    if out is not None and all(len(a) >= m and a.flags.c_contiguous for a in out) and \
            [a.dtype for a in out] == [np.uint64, np.uint64, np.int32, np.int32]:
        ket, bra, re, im = out
    else:
        ket = np.empty(max(m, 1), dtype=np.uint64)
        bra = np.empty(max(m, 1), dtype=np.uint64)
        re = np.empty(max(m, 1), dtype=np.int32)
        im = np.empty(max(m, 1), dtype=np.int32)
    _check(call(_p(ket, C.c_uint64), _p(bra, C.c_uint64), _p(re, C.c_int32), _p(im, C.c_int32), m, C.byref(n)),
           what)
    return ket[:m], bra[:m], re[:m], im[:m]


def ddqmc_import_walkers(run, ket, bra, re, im, t, S, variable=0, q_prev=1, t_var=-1, t_eq=-1):
    ket = np.ascontiguousarray(ket, dtype=np.uint64)
    bra = np.ascontiguousarray(bra, dtype=np.uint64)
    re = np.ascontiguousarray(re, dtype=np.int32)
    im = np.ascontiguousarray(im, dtype=np.int32)
    rc = load().ddqmc_import_walkers(run, _p(ket, C.c_uint64), _p(bra, C.c_uint64), _p(re, C.c_int32),
                                     _p(im, C.c_int32), len(ket), int(t), float(S), int(variable),
                                     int(q_prev), int(t_var), int(t_eq))
    _check(rc, "ddqmc_import_walkers")


def ddqmc_get_state(run):
    s = ddqmc_state()
    _check(load().ddqmc_get_state(run, C.byref(s)), "ddqmc_get_state")
    return s


def ddqmc_get_counts(run):
    r, mc, rc_ = C.c_int64(), C.c_int64(), C.c_int64()
    _check(load().ddqmc_get_counts(run, C.byref(r), C.byref(mc), C.byref(rc_)), "ddqmc_get_counts")
    return r.value, mc.value, rc_.value


def ddqmc_get_totals(run):
    a, b, c, d = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
    _check(load().ddqmc_get_totals(run, C.byref(a), C.byref(b), C.byref(c), C.byref(d)), "ddqmc_get_totals")
    return dict(walker_steps=a.value, entry_steps=b.value, spawn_records=c.value, merged_entries=d.value)


def ddqmc_set_timing(run, enable):
    _check(load().ddqmc_set_timing(run, int(bool(enable))), "ddqmc_set_timing")


def ddqmc_get_timing(run):
    ms = np.zeros(len(KERNEL_CLASSES), dtype=np.float64)
    n = np.zeros(len(KERNEL_CLASSES), dtype=np.int64)
    _check(load().ddqmc_get_timing(run, _p(ms, C.c_double), _p(n, C.c_int64), len(KERNEL_CLASSES)),
           "ddqmc_get_timing")
    return {k: (float(ms[q]), int(n[q])) for q, k in enumerate(KERNEL_CLASSES)}


def ddqmc_wait_selftest(stream=None):
    """Status code of a device wait on a word nothing sets (DDQMC_ERR_TIMEOUT = -5 expected)."""
    return load().ddqmc_wait_selftest(stream)


def ddqmc_annihilate(run, d_list, m, d_spawns, nsp, d_out, out_cap):
    """Device pointers (ints) in and out; returns the merged length."""
    n = C.c_int64()
    _check(load().ddqmc_annihilate(run, C.c_void_p(d_list), int(m), C.c_void_p(d_spawns), int(nsp),
                                   C.c_void_p(d_out), int(out_cap), C.byref(n)), "ddqmc_annihilate")
    return n.value


def ddqmc_annihilate_noalloc(lattice, initiator_threshold, d_list, m, d_spawns, nsp, d_out, out_cap,
                             stream=None):
    """Same as ddqmc_annihilate without a run and without any allocation
    (scratch in a fixed array inside the library); returns the merged length."""
    n = C.c_int64()
    _check(load().ddqmc_annihilate_noalloc(C.byref(lattice), int(initiator_threshold), C.c_void_p(d_list), int(m),
                                           C.c_void_p(d_spawns), int(nsp), C.c_void_p(d_out), int(out_cap),
                                           C.byref(n), C.c_void_p(stream) if stream else None),
           "ddqmc_annihilate_noalloc")
    return n.value


def ddqmc_create_batch(lattice, specs, guide=None, options=None):
    """specs: a sequence of ddqmc_run_spec (one per run)."""
    lib = load()
    arr = (ddqmc_run_spec * len(specs))(*specs)
    h = C.c_void_p()
    rc = lib.ddqmc_create_batch(C.byref(lattice), len(specs), arr, C.byref(guide) if guide is not None else None,
                                C.byref(options) if options is not None else None, C.byref(h))
    _check(rc, "ddqmc_create_batch")
    return h


def ddqmc_batch_estimators(batch, k):
    e = ddqmc_estimates()
    rc = load().ddqmc_batch_estimators(batch, int(k), C.byref(e))
    return rc, e


def ddqmc_batch_raw_estimators(batch, k, cap=1024):
    out = np.zeros(cap, dtype=np.int64)
    n = C.c_int32()
    _check(load().ddqmc_batch_raw_estimators(batch, int(k), _p(out, C.c_int64), cap, C.byref(n)),
           "ddqmc_batch_raw_estimators")
    return out[: n.value]


def ddqmc_tune(run):
    """Autotune the launch shapes on the run's current list (state restored); returns the chosen shapes."""
    t = ddqmc_tuning()
    _check(load().ddqmc_tune(run, C.byref(t)), "ddqmc_tune")
    return t.as_dict()


def ddqmc_get_tuning(run):
    t = ddqmc_tuning()
    _check(load().ddqmc_get_tuning(run, C.byref(t)), "ddqmc_get_tuning")
    return t.as_dict()


def ddqmc_set_tuning(run, **shapes):
    """Change some launch shapes (keyword names of ddqmc_tuning), keeping the others."""
    t = ddqmc_tuning()
    _check(load().ddqmc_get_tuning(run, C.byref(t)), "ddqmc_get_tuning")
    for k, v in shapes.items():
        setattr(t, k, v)
    _check(load().ddqmc_set_tuning(run, C.byref(t)), "ddqmc_set_tuning")


def ddqmc_batch_retire(batch, k):
    """Stop run k of a batch: its walkers leave the list at the next step."""
    _check(load().ddqmc_batch_retire(batch, int(k)), "ddqmc_batch_retire")


def ddqmc_batch_get_state(batch, k):
    s = ddqmc_state()
    _check(load().ddqmc_batch_get_state(batch, int(k), C.byref(s)), "ddqmc_batch_get_state")
    return s


def ddqmc_destroy(run):
    load().ddqmc_destroy(run)


def ddqmc_strerror(code):
    return load().ddqmc_strerror(int(code)).decode()


class Run:
    """One DDQMC run on the GPU (all device memory owned by the library)."""

    def __init__(self, Lx, Ly, periodic, Jx, Jy, Jz, gamma, dt, target, n_a=0, guide_kind=0,
                 guide_p=0.0, site_ratio=None, seed=1, damping=0.05, shift0=-1.0, n0=1000, control=0,
                 t_eq=-1, capacity_entries=0, capacity_spawns=0, stream=None, sm_limit=0, field_h=0.0,
                 field_axis=0, wide_sort_bits=64, field_theta=0.0):
        o = ddqmc_default_options()
        o.seed = int(seed) & ((1 << 64) - 1)
        o.damping = damping
        o.shift0 = shift0
        o.n0 = int(n0)
        o.control = int(control)
        o.t_eq = int(t_eq)
        o.capacity_entries = int(capacity_entries)
        o.capacity_spawns = int(capacity_spawns)
        o.cuda_stream = stream
        o.sm_limit = int(sm_limit)
        o.field_h = float(field_h)
        o.field_axis = int(field_axis)
        o.wide_sort_bits = int(wide_sort_bits)
        o.field_theta = float(field_theta)
        g = ddqmc_guide()
        g.kind = int(guide_kind)
        g.p = float(guide_p)
        self._site_r = None
        if site_ratio is not None:
            self._site_r = np.ascontiguousarray(site_ratio, dtype=np.float64)
            g.site_ratio = _p(self._site_r, C.c_double)
        lat = ddqmc_lattice(int(Lx), int(Ly), int(periodic))
        self.h = ddqmc_create(lat, float(Jx), float(Jy), float(Jz), float(gamma), float(dt), int(target),
                              int(n_a), g, o)
        self.N = Lx * Ly

    def close(self):
        if getattr(self, "h", None):
            ddqmc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n=1):
        _check(ddqmc_step(self.h, n), "ddqmc_step")

    def step_async(self, n=1):
        _check(ddqmc_step_async(self.h, n), "ddqmc_step_async")

    def sync(self):
        _check(ddqmc_sync(self.h), "ddqmc_sync")

    def estimates(self):
        rc, e = ddqmc_estimators(self.h)
        _check(rc, "ddqmc_estimators")
        return e

    def raw_estimates(self):
        return ddqmc_raw_estimators(self.h)

    def export(self, out=None):
        return ddqmc_export_walkers(self.h, out)

    def import_(self, ket, bra, re, im, t, S, variable=0, q_prev=1, t_var=-1, t_eq=-1):
        ddqmc_import_walkers(self.h, ket, bra, re, im, t, S, variable, q_prev, t_var, t_eq)

    def export_records(self, out=None):
        return ddqmc_export_records(self.h, out)

    def import_records(self, recs, t, S, variable=0, q_prev=1, t_var=-1, t_eq=-1):
        ddqmc_import_records(self.h, recs, t, S, variable, q_prev, t_var, t_eq)

    def export_records32(self, out=None):
        return ddqmc_export_records32(self.h, out)

    def import_records32(self, recs, t, S, variable=0, q_prev=1, t_var=-1, t_eq=-1):
        ddqmc_import_records32(self.h, recs, t, S, variable, q_prev, t_var, t_eq)

    def state(self):
        return ddqmc_get_state(self.h)

    def counts(self):
        return ddqmc_get_counts(self.h)

    def tune(self):
        return ddqmc_tune(self.h)

    def tuning(self):
        return ddqmc_get_tuning(self.h)


def run_spec(Jx, Jy, Jz, gamma, dt, target, n_a=0, seed=1, damping=0.05, shift0=-1.0, n0=1000, control=0,
             t_eq=-1, field_h=0.0, field_axis=0, field_theta=0.0):
    """A ddqmc_run_spec with the keyword names of ``Run``."""
    q = ddqmc_run_spec()
    q.Jx, q.Jy, q.Jz, q.gamma, q.dt = float(Jx), float(Jy), float(Jz), float(gamma), float(dt)
    q.target_walkers = int(target)
    q.initiator_threshold = int(n_a)
    q.control = int(control)
    q.seed = int(seed) & ((1 << 64) - 1)
    q.damping = float(damping)
    q.shift0 = float(shift0)
    q.n0 = int(n0)
    q.t_eq = int(t_eq)
    q.field_h = float(field_h)
    q.field_axis = int(field_axis)
    q.reserved = 0
    q.field_theta = float(field_theta)
    return q


class Batch:
    """Several DDQMC runs of one lattice stepped together in one walker store
    (run id in the key's high bits); runs[k] are the keyword arguments of
    ``run_spec`` for run k.  ``wide_sort_bits``: the key order of two-word
    keys, as for ``Run`` (the run id sits above the hash bits)."""

    def __init__(self, Lx, Ly, periodic, runs, guide_kind=0, guide_p=0.0, site_ratio=None,
                 capacity_entries=0, capacity_spawns=0, stream=None, sm_limit=0, wide_sort_bits=64):
        o = ddqmc_default_options()
        o.capacity_entries = int(capacity_entries)
        o.capacity_spawns = int(capacity_spawns)
        o.wide_sort_bits = int(wide_sort_bits)
        o.cuda_stream = stream
        o.sm_limit = int(sm_limit)
        g = ddqmc_guide()
        g.kind = int(guide_kind)
        g.p = float(guide_p)
        self._site_r = None
        if site_ratio is not None:
            self._site_r = np.ascontiguousarray(site_ratio, dtype=np.float64)
            g.site_ratio = _p(self._site_r, C.c_double)
        specs = [run_spec(**r) for r in runs]
        self.h = ddqmc_create_batch(ddqmc_lattice(int(Lx), int(Ly), int(periodic)), specs, g, o)
        self.nruns = len(specs)
        self.N = Lx * Ly

    def close(self):
        if getattr(self, "h", None):
            ddqmc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n=1):
        _check(ddqmc_step(self.h, n), "ddqmc_step")

    def step_async(self, n=1):
        _check(ddqmc_step_async(self.h, n), "ddqmc_step_async")

    def sync(self):
        _check(ddqmc_sync(self.h), "ddqmc_sync")

    def estimates(self, k):
        rc, e = ddqmc_batch_estimators(self.h, k)
        _check(rc, "ddqmc_batch_estimators")
        return e

    def raw_estimates(self, k):
        return ddqmc_batch_raw_estimators(self.h, k)

    def export(self, k, out=None):
        return ddqmc_batch_export_walkers(self.h, k, out)

    def state(self, k):
        return ddqmc_batch_get_state(self.h, k)

    def retire(self, k):
        ddqmc_batch_retire(self.h, k)

    def tune(self):
        return ddqmc_tune(self.h)

    def totals(self):
        return ddqmc_get_totals(self.h)
