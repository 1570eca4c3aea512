"""Single-step transitions worked by hand, with an injected uniform stream in
place of Philox (four 32-bit words per walker block, in the order the step
draws them).  Numbers below were computed by hand from the written rules:
rates q(x) = trunc(x * 2^32), ket moves before bra moves before jumps,
death p = dt((gamma/2)(n(i)+n(j)) + S), cross q = dt |Jz| |zsum(i) - zsum(j)|.
"""
import numpy as np

from oracle import oracle as O

FULL = 0xFFFFFFFF


def _list(run):
    k, b, r, i = run.export()
    return [(int(a), int(c), int(x), int(y)) for a, c, x, y in zip(k, b, r, i)]


def _run(Lx, Ly, dt, S, n_a=0, Jx=0.9, Jy=1.0, Jz=1.0, gamma=1.0):
    run = O.OracleRun(Lx, Ly, 0, Jx, Jy, Jz, gamma, dt, 10 ** 15, n_a=n_a, shift0=S)
    return run


def test_two_site_ket_spawn_and_clone():
    # 2-site chain, one real walker on |dd><dd|.  Both moves act on an aligned
    # bond: rate 0.1 * 0.01 * 2^32 = 4294967.296 -> 4294967 each; T = 8589934.
    # Death: p = 0.01 * (0 + S) = -0.01 (cloning), threshold 42949672.
    run = _run(2, 1, 0.01, -1.0)
    run.import_([0], [0], [1], [0])
    run.inject([100, 0, 0, 0])           # ket move (100 < 4294967); clone (0 < 42949672)
    run.step(1)
    # ket move: child (3, 0), A = -i (Jx - Jy) = +0.1 i -> imaginary child, sign +
    assert _list(run) == [(0, 0, 2, 0), (3, 0, 0, 1)]
    assert run.injected_used() == 4


def test_two_site_bra_spawn_no_clone():
    run = _run(2, 1, 0.01, -1.0)
    run.import_([0], [0], [1], [0])
    run.inject([5000000, 42949672, 0, 0])  # bra move (4294967 <= u < 8589934); no clone
    run.step(1)
    # bra move: child (0, 3), A = +i (Jx - Jy) = -0.1 i -> imaginary child, sign -
    assert _list(run) == [(0, 0, 1, 0), (0, 3, 0, -1)]


def test_two_site_no_spawn_at_total_rate():
    run = _run(2, 1, 0.01, -1.0)
    run.import_([0], [0], [1], [0])
    run.inject([8589934, 42949671, 0, 0])  # u = T: no spawn; u < 42949672: clone
    run.step(1)
    assert _list(run) == [(0, 0, 2, 0)]


def test_four_attempts_deterministic_death_and_cross():
    # 2-site chain, dt = 2, S = 0, one real walker on (ket 1, bra 0).
    # ket bond anti-aligned: q(1.9 * 2) = trunc(16320875724.8) = 16320875724
    # bra bond aligned:      q(0.1 * 2) = trunc(858993459.2)   = 858993459
    # T = 17179869183 -> n_att = ceil(T / 2^32) = 4, v = 4u.
    # death c = 1: p = 2 * 0.5 = 1.0 -> exactly one death, no random part.
    # cross: zsum(1) = -1, zsum(0) = +1, q = 2 * 1 * 2 = 4 -> 4 walkers Re -> Im,
    #        d = -Jz (zsum(i) - zsum(j)) = +2 > 0, so +4 on Im.
    run = _run(2, 1, 2.0, 0.0)
    run.import_([1], [0], [1], [0])
    run.inject([0, 0, 0, FULL,                  # block 0: attempt 0 -> ket; attempt 1 (v = 4u = 17179869180 < T) -> bra
                0xF0000000, 0xFF000000, 0, 0])  # block 1: attempt 2 -> ket (v < 16320875724); attempt 3 -> bra
    run.step(1)
    assert run.injected_used() == 8
    # ket children (2, 0): A = -1.9 i -> Im, sign -; bra children (1, 3): A = -0.1 i -> Im, sign -
    assert _list(run) == [(1, 0, 0, 4), (2, 0, 0, -2), (1, 3, 0, -2)]


def test_initiator_drops_child_on_empty_offdiagonal():
    # 3-site open chain, n_a = 3; (ket 3, bra 0) holds one imaginary walker, so it
    # is not an initiator.  Rates (dt = 0.01): ket b0 aligned 4294967, ket b1
    # anti 81604378 (1.9 * 0.01 * 2^32 = 81604378.624), bra b0, b1 aligned
    # 4294967 each; cumulative 4294967, 85899345, 90194312, 94489279.
    # u0 = 50000000 selects ket b1: child (5, 0), A = -1.9 i; imaginary parent
    # -> real child with sign -sgn(Im A) = +1.  (5, 0) is empty and off-diagonal:
    # the child is dropped.  Death (c = 2, S = 0): p = 0.01, threshold 42949672;
    # cross: zsum(3) = 0, zsum(0) = 2, q = 0.02 -> threshold 85899345, d = +2.
    run = _run(3, 1, 0.01, 0.0, n_a=3)
    run.import_([3], [0], [0], [1])
    run.inject([50000000, FULL, FULL, FULL])
    run.step(1)
    assert _list(run) == [(3, 0, 0, 1)]


def test_initiator_keeps_child_on_occupied_target():
    # as above, with (5, 0) occupied by two real walkers that neither spawn,
    # die nor transfer (all-ones words); the non-initiator child now survives.
    run = _run(3, 1, 0.01, 0.0, n_a=3)
    run.import_([3, 5], [0, 0], [0, 2], [1, 0])
    run.inject([50000000, FULL, 0, FULL,       # (3,0) Im walker: ket b1 child; cross fires (0 < 85899345)
                FULL, FULL, FULL, FULL,        # (5,0) Re walker 0
                FULL, FULL, FULL, FULL])       # (5,0) Re walker 1
    run.step(1)
    # cross on the imaginary walker moves one walker to Re with sign -sgn(d) = -1
    assert _list(run) == [(3, 0, -1, 1), (5, 0, 3, 0)]


def test_initiator_keeps_child_on_diagonal():
    # u0 = 1000 selects ket b0: child (0, 0), diagonal, so it always survives.
    # A = -i (Jx - Jy) = +0.1 i, imaginary parent -> real child, sign -sgn(0.1) = -1
    run = _run(3, 1, 0.01, 0.0, n_a=3)
    run.import_([3], [0], [0], [1])
    run.inject([1000, FULL, FULL, FULL])
    run.step(1)
    assert _list(run) == [(0, 0, -1, 0), (3, 0, 0, 1)]


def test_move_groups_order_aligned_before_anti_aligned():
    # 3-site open chain, one real walker on (ket 1, bra 1): in ket 1 (site 0 up)
    # bond b0 = (0,1) is anti-aligned and b1 = (1,2) aligned, so the ket moves
    # come as b1 (aligned group) then b0 (anti-aligned group), although b0
    # comes first in bond order; the same holds for the bra moves.
    # dt = 0.01: aligned rate 0.1*0.01*2^32 -> 4294967, anti-aligned
    # 1.9*0.01*2^32 -> 81604378; cumulative ket: 4294967, 85899345.
    # u0 = 1000 < 4294967 selects the ket move on b1: child (1 ^ 6, 1) = (7, 1),
    # A = -i (Jx - Jy) = +0.1 i -> imaginary child, sign +.
    # Death (c = 2, S = 0): p = 0.01; all-ones words: no death, no transfer.
    run = _run(3, 1, 0.01, 0.0)
    run.import_([1], [1], [1], [0])
    run.inject([1000, FULL, FULL, FULL])
    run.step(1)
    assert _list(run) == [(1, 1, 1, 0), (7, 1, 0, 1)]
    # u0 = 4294967 selects the first anti-aligned move: b0, child (1 ^ 3, 1) = (2, 1),
    # A = -i (Jx + Jy) = -1.9 i -> imaginary child, sign -.
    run = _run(3, 1, 0.01, 0.0)
    run.import_([1], [1], [1], [0])
    run.inject([4294967, FULL, FULL, FULL])
    run.step(1)
    assert _list(run) == [(1, 1, 1, 0), (2, 1, 0, -1)]
