"""Two-word keys (more than 31 sites) in the hashed order: the spawn records
are sorted on the stored bra word only (bra xor a hash of the ket), and a
repair kernel puts records that share it in ket order.  The order is internal:
lists, estimators and the step must equal the oracle's bit for bit whatever
the number of hash bits, for single runs and batches, and import / export
keep the caller's (bra, ket) order."""
import numpy as np
import pytest

from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ddqmc():
    import __graft_entry__ as g
    g.build()
    from paper_1802_05931_gb300 import ddqmc as d
    return d


def _same(gpu, cpu, where):
    g = gpu.export()
    c = cpu.export()
    assert len(g[0]) == len(c[0]), (where, len(g[0]), len(c[0]))
    for name, a, b in zip(("ket", "bra", "re", "im"), g, c):
        assert np.array_equal(a, b), (where, name)
    assert np.array_equal(gpu.raw_estimates(), cpu.estimates_now()), where


@pytest.mark.parametrize("bits", [64, 0, 3, -1])
def test_sort_orders_bitexact(ddqmc, bits):
    """6x6 periodic: the default 64 hash bits; none (every stored bra word is
    the bra word, so each step repairs one group per bra with several kets);
    3 bits; and the plain order on every key bit."""
    args = (6, 6, 1, 0.9, 1.0, 1.0, 1.0, 0.005, 2000)
    kw = dict(n_a=3, control=1, seed=5)
    gpu = ddqmc.Run(*args, wide_sort_bits=bits, capacity_entries=1 << 18, capacity_spawns=1 << 19, **kw)
    cpu = O.OracleRun(*args, **kw)
    for t in range(80):
        gpu.step(1)
        cpu.step(1)
        if t % 4 == 0 or t >= 77:
            _same(gpu, cpu, (bits, t))
    assert gpu.export()[0].size > 300


def test_hashed_8x8_graph_steps(ddqmc):
    """8x8 periodic in the hashed order (the default 64 bits: 8 digit passes
    instead of 16), stepped by captured graphs of 32 steps, against the
    oracle."""
    args = (8, 8, 1, 0.9, 1.0, 1.0, 1.0, 0.005, 5000)
    kw = dict(n_a=3, control=1, seed=9)
    gpu = ddqmc.Run(*args, capacity_entries=1 << 20, capacity_spawns=1 << 21, **kw)
    cpu = O.OracleRun(*args, **kw)
    for n in (33, 31):
        gpu.step(n)
        cpu.step(n)
        _same(gpu, cpu, n)


@pytest.mark.parametrize("bits,nbra,nket", [(4, 16, 40), (1, 2, 3000)])
def test_import_export_roundtrip(ddqmc, bits, nbra, nket):
    """Import sorts a (bra, ket)-ordered list into the hashed order (groups of
    equal stored bra words mix bra words, so their kets arrive out of order:
    small groups sort in shared memory, groups of about 3000 entries in
    place); export sorts it back.  Then a few steps from the imported list
    equal the plain order's (few hash bits give many groups to repair in every
    step, so the populations are small)."""
    rng = np.random.default_rng(bits)
    N = 36
    # bra words that differ only in the hashed bits: every group of equal
    # stored words holds entries of every bra word
    base = int(rng.integers(0, 1 << (N - bits))) << bits
    bras = (base | np.arange(nbra)).astype(np.uint64)
    kets = np.sort(rng.choice(1 << N, size=nket, replace=False)).astype(np.uint64)
    bra = np.repeat(bras, nket)
    ket = np.tile(kets, nbra)
    re = rng.integers(-3, 4, size=bra.size).astype(np.int32)
    im = rng.integers(-3, 4, size=bra.size).astype(np.int32)
    re[(re == 0) & (im == 0)] = 1
    run = ddqmc.Run(6, 6, 1, 0.9, 1.0, 1.0, 1.0, 0.005, 10 ** 5, n_a=3, control=1, seed=2, wide_sort_bits=bits,
                    capacity_entries=1 << 16, capacity_spawns=1 << 16)
    run.import_(ket, bra, re, im, 0, -1.0, 0, 0, 0, 0)
    k2, b2, r2, i2 = run.export()
    for a, b in ((k2, ket), (b2, bra), (r2, re), (i2, im)):
        assert np.array_equal(a, b)
    # and it steps like the plain order
    plain = ddqmc.Run(6, 6, 1, 0.9, 1.0, 1.0, 1.0, 0.005, 10 ** 5, n_a=3, control=1, seed=2, wide_sort_bits=-1,
                      capacity_entries=1 << 18, capacity_spawns=1 << 19)
    plain.import_(ket, bra, re, im, 0, -1.0, 0, 0, 0, 0)
    run2 = ddqmc.Run(6, 6, 1, 0.9, 1.0, 1.0, 1.0, 0.005, 10 ** 5, n_a=3, control=1, seed=2, wide_sort_bits=bits,
                     capacity_entries=1 << 18, capacity_spawns=1 << 19)
    run2.import_(ket, bra, re, im, 0, -1.0, 0, 0, 0, 0)
    for _ in range(3):
        plain.step(1)
        run2.step(1)
        for a, b in zip(plain.export(), run2.export()):
            assert np.array_equal(a, b)
        assert np.array_equal(plain.raw_estimates(), run2.raw_estimates())


@pytest.mark.parametrize("bits", [0, 3, 50])
def test_batch_hashed_order_against_the_oracle(ddqmc, bits):
    """A 6x6 batch in the hashed order, against the oracle run by run, after
    single steps and after graph blocks; then a retired run.  Few hash bits
    leave many groups of equal stored bra words to repair in every step (the
    run id above the 36 spin bits keeps the runs' groups apart); 50 bits are
    capped at 46 (one digit byte past the spin and run-id bits), which puts
    the run id above the hash, at bit 46."""
    # at most about 9,000 spawn records per step in all: fewer out-of-order
    # neighbours than the repair records, whatever the order
    runs = [dict(Jx=(0.8, 0.9, 1.15)[k], Jy=1.0, Jz=1.0, gamma=1.0, dt=0.005, target=1500 + 500 * k, n_a=3,
                 seed=40 + k, control=1) for k in range(3)]
    batch = ddqmc.Batch(6, 6, 1, runs, capacity_entries=1 << 18, capacity_spawns=1 << 19, wide_sort_bits=bits)
    cpus = [O.OracleRun(6, 6, 1, r["Jx"], r["Jy"], r["Jz"], r["gamma"], r["dt"], r["target"], n_a=r["n_a"],
                        seed=r["seed"], control=r["control"]) for r in runs]
    for t in (1, 2, 3, 10, 40, 73):
        done = batch.state(0).t
        batch.step(t - done)
        for k, cpu in enumerate(cpus):
            cpu.step(t - done)
            g, c = batch.export(k), cpu.export()
            assert len(g[0]) == len(c[0]), (bits, t, k)
            for name, a, b in zip(("ket", "bra", "re", "im"), g, c):
                assert np.array_equal(a, b), (bits, t, k, name)
            assert np.array_equal(batch.raw_estimates(k), cpu.estimates_now()), (bits, t, k)
    assert all(batch.export(k)[0].size > 1000 for k in range(len(runs)))
    # run 1 retires: its entries leave at the next merge, the others go on
    batch.retire(1)
    batch.step(5)
    assert batch.export(1)[0].size == 0
    for k in (0, 2):
        cpus[k].step(5)
        for a, b in zip(batch.export(k), cpus[k].export()):
            assert np.array_equal(a, b), (bits, "retired", k)


def test_invalid_sort_bits(ddqmc):
    for bits in (-2, 65):
        with pytest.raises(ddqmc.DDQMCError):
            ddqmc.Run(6, 6, 1, 0.9, 1.0, 1.0, 1.0, 0.005, 1000, wide_sort_bits=bits)
