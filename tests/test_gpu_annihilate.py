"""ddqmc_annihilate (onesweep radix sort + merge-path merge on caller-provided
device records) against the oracle's annihilation, bit for bit."""
import numpy as np
import pytest

from oracle import oracle as O
from tests import records as RC

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_1802_05931_gb300 import ddqmc
    return torch, ddqmc


def _dev(torch, recs):
    b = np.ascontiguousarray(recs).view(np.uint8)
    t = torch.from_numpy(b.copy()).cuda() if len(b) else torch.empty(16, dtype=torch.uint8, device="cuda")
    return t


def run_case(env, run, N, n_a, L, S):
    torch, ddqmc = env
    dl, ds = _dev(torch, L), _dev(torch, S)
    cap = len(L) + len(S) + 1
    out = torch.empty(cap * 16, dtype=torch.uint8, device="cuda")
    n = ddqmc.ddqmc_annihilate(run.h, dl.data_ptr(), len(L), ds.data_ptr(), len(S), out.data_ptr(), cap)
    got = out[: n * 16].cpu().numpy().view(RC.REC)
    lk, lb, lr, li, _ = RC.split(L, N)
    sk, sb, sr, si, sf = RC.split(S, N)
    ok, ob, orr, oi = O.annihilate(lk, lb, lr, li, sk, sb, sr, si, sf, n_a)
    ref = np.zeros(len(ok), dtype=RC.REC)
    ref["key"] = (ob << np.uint64(N)) | ok
    ref["re"] = orr
    ref["im"] = oi
    return got, ref


@pytest.mark.parametrize("n_a", [0, 3])
@pytest.mark.parametrize("m,r", [(0, 0), (0, 7), (5, 0), (1, 1), (3000, 5000), (2047, 2049), (40000, 100000),
                                 (250000, 700000)])
def test_annihilate_matches_oracle(env, n_a, m, r):
    torch, ddqmc = env
    N = 16
    run = ddqmc.Run(4, 4, 1, 0.9, 1.0, 1.0, 1.0, 0.005, 10 ** 6, n_a=n_a, control=1,
                    capacity_entries=1 << 21, capacity_spawns=1 << 21)
    L, S = RC.random_case(1000 * m + r + n_a, N, m, r)
    got, ref = run_case(env, run, N, n_a, L, S)
    assert len(got) == len(ref)
    assert np.array_equal(got["key"], ref["key"])
    assert np.array_equal(got["re"], ref["re"]) and np.array_equal(got["im"], ref["im"])


def test_annihilate_twice_in_a_row_and_between_steps(env):
    """Standalone calls interleaved with steps of the same run give the same
    results and leave the run's own stepping untouched."""
    torch, ddqmc = env
    N = 9
    args = (3, 3, 1, 0.9, 1.0, 1.0, 1.0, 0.005, 20000)
    run = ddqmc.Run(*args, n_a=3, control=1)
    ref_run = O.OracleRun(*args, n_a=3, control=1)
    L, S = RC.random_case(5, N, 20000, 60000)
    first = run_case(env, run, N, 3, L, S)
    for _ in range(3):
        run.step(40)
        ref_run.step(40)
        got, ref = run_case(env, run, N, 3, L, S)
        assert np.array_equal(got, first[0]) and np.array_equal(got, ref)
    g = run.export()
    c = ref_run.export()
    for a, b in zip(g, c):
        assert np.array_equal(a, b)


def test_annihilate_rejects_too_many_spawns(env):
    torch, ddqmc = env
    run = ddqmc.Run(2, 2, 0, 0.9, 1.0, 1.0, 1.0, 0.01, 100, capacity_entries=4096, capacity_spawns=4096)
    x = torch.empty(16 * 8192, dtype=torch.uint8, device="cuda")
    with pytest.raises(ddqmc.DDQMCError) as e:
        ddqmc.ddqmc_annihilate(run.h, x.data_ptr(), 0, x.data_ptr(), 8192, x.data_ptr(), 8192)
    assert e.value.code == -3


def test_annihilate_rejects_two_word_keys(env):
    """The 16-byte records of the standalone annihilation hold one-word keys
    (N <= 31); a run with more sites is refused, not misread."""
    torch, ddqmc = env
    run = ddqmc.Run(6, 6, 1, 0.9, 1.0, 1.0, 1.0, 0.005, 100)
    x = torch.empty(16 * 64, dtype=torch.uint8, device="cuda")
    with pytest.raises(ddqmc.DDQMCError) as e:
        ddqmc.ddqmc_annihilate(run.h, x.data_ptr(), 1, x.data_ptr(), 1, x.data_ptr(), 64)
    assert e.value.code == -7          # DDQMC_ERR_UNSUPPORTED


@pytest.mark.parametrize("part,sign", [("re", 1), ("re", -1), ("im", 1)])
def test_annihilate_int32_overflow_is_reported(env, part, sign):
    """A list entry 10 walkers short of the int32 limit that receives 20 more
    through its spawn records leaves the int32 range: the call reports
    DDQMC_ERR_OVERFLOW instead of a wrapped population, and the oracle's
    annihilation reports its overflow code on the same arrays.  A following
    call on the same run with valid records succeeds."""
    torch, ddqmc = env
    N = 16
    run = ddqmc.Run(4, 4, 1, 0.9, 1.0, 1.0, 1.0, 0.005, 10 ** 6, n_a=3, control=1,
                    capacity_entries=1 << 16, capacity_spawns=1 << 16)
    L = np.zeros(3, dtype=RC.REC)
    L["key"] = np.array([5, (7 << N) | 3, (9 << N) | 9], dtype=np.uint64)
    L["re"] = [1, 0, -2]
    L["im"] = [0, 0, 1]
    L[part][1] = sign * (2 ** 31 - 10)
    S = np.zeros(6, dtype=RC.REC)
    S["key"] = np.uint64((7 << N) | 3) | RC.FLAG
    S[part] = sign * 4
    S["key"][5] = np.uint64(11 << N | 2)         # an unrelated record
    S[part][5] = 0
    S["re"][5] = 1
    dl, ds = _dev(torch, L), _dev(torch, S)
    out = torch.empty(16 * 16, dtype=torch.uint8, device="cuda")
    with pytest.raises(ddqmc.DDQMCError) as e:
        ddqmc.ddqmc_annihilate(run.h, dl.data_ptr(), len(L), ds.data_ptr(), len(S), out.data_ptr(), 16)
    assert e.value.code == -4                     # DDQMC_ERR_OVERFLOW
    lk, lb, lr, li, _ = RC.split(L, N)
    sk, sb, sr, si, sf = RC.split(S, N)
    with pytest.raises(RuntimeError, match=r"\(-4\)"):
        O.annihilate(lk, lb, lr, li, sk, sb, sr, si, sf, 3)
    # the same entry with records summing to +4 stays in range
    S[part][3] = -sign * 4
    S[part][4] = -sign * 4
    got, ref = run_case(env, run, N, 3, L, S)
    assert np.array_equal(got, ref)
    k = np.nonzero(got["key"] == np.uint64((7 << N) | 3))[0][0]
    assert int(got[part][k]) == sign * (2 ** 31 - 6)


def test_annihilate_rejects_misaligned_records(env):
    """16-byte records are moved with 16-byte accesses and bulk copies: a
    record pointer that is not 16-byte aligned is refused on the host before
    any launch."""
    torch, ddqmc = env
    run = ddqmc.Run(4, 4, 1, 0.9, 1.0, 1.0, 1.0, 0.005, 10 ** 4, capacity_entries=4096, capacity_spawns=4096)
    x = torch.zeros(16 * 64 + 64, dtype=torch.uint8, device="cuda")
    p = x.data_ptr()
    assert p % 16 == 0
    for args in ((p + 8, 1, p, 1, p + 512, 8), (p, 1, p + 4, 1, p + 512, 8), (p, 1, p, 1, p + 520, 8)):
        with pytest.raises(ddqmc.DDQMCError) as e:
            ddqmc.ddqmc_annihilate(run.h, *args)
        assert e.value.code == -1      # DDQMC_ERR_INVALID_ARG
