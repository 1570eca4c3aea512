"""The allocation-free annihilation entry point against the ordinary one.

ddqmc_annihilate_noalloc exists for callers that cannot call cudaMalloc:
code running inside a process whose device memory is already reserved by
another allocator's pool, or loops that must stay off the driver's
allocation path.  It keeps its scratch in a fixed array inside the library.
This test calls it through the C-ABI, twice in a row, and requires the same
merged list as ddqmc_annihilate (which uses a run's allocated buffers) on the
same inputs, bit for bit as for every integer result in this suite.  It sits
in the file collected last so that a failure here cannot hide another test.
"""
import numpy as np
import pytest

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
    if len(b) == 0:
        return torch.empty(16, dtype=torch.uint8, device="cuda")
    return torch.from_numpy(b.copy()).cuda()


@pytest.mark.parametrize("Lx,Ly,per,n_a,m,r", [(4, 4, 1, 3, 200000, 250000), (3, 3, 1, 0, 30000, 262144)])
def test_noalloc_matches_allocating_entry_point_twice(env, Lx, Ly, per, n_a, m, r):
    torch, ddqmc = env
    N = Lx * Ly
    run = ddqmc.Run(Lx, Ly, per, 0.9, 1.0, 1.0, 1.0, 0.005, 10 ** 5, n_a=n_a, control=1,
                    capacity_entries=1 << 21, capacity_spawns=1 << 21)
    L, S = RC.random_case(77 + m, N, m, r)
    dl, ds = _dev(torch, L), _dev(torch, S)
    cap = len(L) + len(S) + 1
    ref = torch.empty(cap * 16, dtype=torch.uint8, device="cuda")
    n_ref = ddqmc.ddqmc_annihilate(run.h, dl.data_ptr(), len(L), ds.data_ptr(), len(S), ref.data_ptr(), cap)
    ref_h = ref[: n_ref * 16].cpu().numpy()
    lat = ddqmc.ddqmc_lattice(Lx, Ly, per)
    for _ in range(2):
        out = torch.full((cap * 16,), 0xAB, dtype=torch.uint8, device="cuda")
        n = ddqmc.ddqmc_annihilate_noalloc(lat, n_a, dl.data_ptr(), len(L), ds.data_ptr(), len(S),
                                           out.data_ptr(), cap)
        assert n == n_ref
        assert np.array_equal(out[: n * 16].cpu().numpy(), ref_h)


def test_noalloc_rejects_sizes_beyond_its_maximum(env):
    torch, ddqmc = env
    x = torch.empty(16, dtype=torch.uint8, device="cuda")
    lat = ddqmc.ddqmc_lattice(4, 4, 1)
    with pytest.raises(ddqmc.DDQMCError) as e:
        ddqmc.ddqmc_annihilate_noalloc(lat, 3, x.data_ptr(), 0, x.data_ptr(), ddqmc.NOALLOC_MAX_SPAWNS + 1,
                                       x.data_ptr(), 1)
    assert e.value.code == -3
    with pytest.raises(ddqmc.DDQMCError) as e:
        ddqmc.ddqmc_annihilate_noalloc(lat, 3, x.data_ptr(), ddqmc.NOALLOC_MAX_LIST + 1, x.data_ptr(), 0,
                                       x.data_ptr(), 1)
    assert e.value.code == -3
