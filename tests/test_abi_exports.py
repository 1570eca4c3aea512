"""The C-ABI library builds, loads without a GPU and exports every entry point
that include/ddqmc.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    with open(os.path.join(ROOT, "include", "ddqmc.h")) as f:
        text = f.read()
    for m in re.finditer(r"^(?:int|void|const char \*)\s*\*?\s*(ddqmc_\w+)\s*\(", text, re.M):
        names.append(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("ddqmc_create", "ddqmc_step", "ddqmc_estimators", "ddqmc_destroy",
                     "ddqmc_export_walkers", "ddqmc_import_walkers", "ddqmc_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_1802_05931_gb300 import build as b
    path = b.build()
    lib = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_wraps_every_declared_symbol():
    from paper_1802_05931_gb300 import ddqmc
    for name in _declared():
        assert name in ddqmc.EXPORTS and hasattr(ddqmc, name), name


def test_strerror_and_options_need_no_gpu():
    from paper_1802_05931_gb300 import build as b, ddqmc
    b.build()
    assert ddqmc.ddqmc_strerror(-3).startswith("walker list")
    o = ddqmc.ddqmc_default_options()
    assert o.seed == 1 and o.damping == 0.05 and o.shift0 == -1.0 and o.n0 == 1000


def test_option_defaults_and_parameter_checks_need_no_gpu():
    """Defaults of the newer option fields, and parameters that ddqmc_create
    rejects before touching the device."""
    from paper_1802_05931_gb300 import build as b, ddqmc
    b.build()
    o = ddqmc.ddqmc_default_options()
    assert o.sm_limit == 0 and o.field_h == 0.0 and o.field_axis == 0 and o.field_theta == 0.0
    assert o.wide_sort_bits == 64
    lat = ddqmc.ddqmc_lattice(2, 2, 0)
    for lattice, opt in ((ddqmc.ddqmc_lattice(9, 8, 0), None),          # 72 sites
                         (ddqmc.ddqmc_lattice(2, 2, 1), None),          # L = 2 periodic
                         (lat, dict(field_axis=3)),                     # no such axis
                         (lat, dict(field_h=float("nan"))),
                         (lat, dict(field_axis=2, field_theta=float("inf"))),
                         (lat, dict(wide_sort_bits=65)),
                         (lat, dict(control=3))):
        oo = ddqmc.ddqmc_default_options()
        for k, v in (opt or {}).items():
            setattr(oo, k, v)
        with pytest.raises(ddqmc.DDQMCError) as e:
            ddqmc.ddqmc_create(lattice, 0.9, 1.0, 1.0, 1.0, 0.01, 100, 0, None, oo)
        assert e.value.code == -1


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_1802_05931_gb300 import ddqmc
    with pytest.raises(RuntimeError):
        _fresh_load(str(tmp_path / "missing.so"))


def _fresh_load(path):
    from paper_1802_05931_gb300 import ddqmc
    saved = ddqmc._lib
    ddqmc._lib = None
    try:
        ddqmc.load(path)
    finally:
        ddqmc._lib = saved


def test_batch_parameter_checks_need_no_gpu():
    """ddqmc_create_batch rejects what it cannot run before touching the
    device: no runs, too many runs, a bad run parameter, 64 sites (the run id
    would need an extra key word), 31 sites with 3 runs (62 spin bits + 2
    run bits do not fit below the flag bit of a one-word key), 63 sites with
    3 runs (63 + 2 bits do not fit in the bra word), and a bad sort order."""
    from paper_1802_05931_gb300 import build as b, ddqmc
    b.build()
    base = ddqmc.run_spec(0.9, 1.0, 1.0, 1.0, 0.01, 1000)
    bad = ddqmc.run_spec(0.9, 1.0, 1.0, 1.0, 0.0, 1000)
    lat = ddqmc.ddqmc_lattice(2, 2, 0)
    for lattice, specs, code in ((lat, [], -1),
                                 (lat, [base] * (ddqmc.MAX_BATCH + 1), -1),
                                 (lat, [base, bad], -1),
                                 (ddqmc.ddqmc_lattice(8, 8, 1), [base, base], -7),
                                 (ddqmc.ddqmc_lattice(31, 1, 0), [base] * 3, -7),
                                 (ddqmc.ddqmc_lattice(7, 9, 0), [base] * 3, -7)):
        with pytest.raises(ddqmc.DDQMCError) as e:
            ddqmc.ddqmc_create_batch(lattice, specs)
        assert e.value.code == code
    for bits in (-2, 65):
        o = ddqmc.ddqmc_default_options()
        o.wide_sort_bits = bits
        with pytest.raises(ddqmc.DDQMCError) as e:
            ddqmc.ddqmc_create_batch(ddqmc.ddqmc_lattice(6, 6, 1), [base, base], options=o)
        assert e.value.code == -1
