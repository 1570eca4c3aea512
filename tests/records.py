"""Seeded synthetic spawn records and walker lists for the annihilation tests
(16-byte records: uint64 key = bra << N | ket with bit 63 the initiator flag,
int32 re, int32 im).  Generators only: no arithmetic of the method here."""
import numpy as np

REC = np.dtype([("key", "<u8"), ("re", "<i4"), ("im", "<i4")])
FLAG = np.uint64(1) << np.uint64(63)


def random_case(seed, N, m, r, diag_frac=0.05, hit_frac=0.4, zero_frac=0.1):
    rng = np.random.default_rng(seed)
    mask = (1 << N) - 1
    # list: unique sorted keys
    raw = rng.integers(0, 1 << (2 * N), size=int(m * 1.3) + 8, dtype=np.uint64)
    keys = np.unique(raw)[:m]
    rng.shuffle(keys)
    keys = np.sort(keys[:m])
    L = np.zeros(len(keys), dtype=REC)
    L["key"] = keys
    L["re"] = rng.integers(-5, 6, len(keys))
    L["im"] = rng.integers(-5, 6, len(keys))
    L["re"][(L["re"] == 0) & (L["im"] == 0)] = 1
    # spawns: fresh keys, keys of the list, diagonal keys; repeated keys
    S = np.zeros(r, dtype=REC)
    fresh = rng.integers(0, 1 << (2 * N), size=r, dtype=np.uint64)
    if len(keys):
        hit = keys[rng.integers(0, len(keys), size=r)]
        fresh = np.where(rng.random(r) < hit_frac, hit, fresh)
    d = rng.integers(0, 1 << N, size=r, dtype=np.uint64)
    diag = (d << np.uint64(N)) | d
    fresh = np.where(rng.random(r) < diag_frac, diag, fresh)
    # repeat some keys many times (runs longer than a tile)
    if r > 10:
        fresh[rng.integers(0, r, size=r // 20)] = fresh[0]
    S["key"] = fresh
    S["re"] = rng.integers(-2, 3, r)
    S["im"] = rng.integers(-2, 3, r)
    zero = rng.random(r) < zero_frac
    S["re"][zero] = 0
    S["im"][zero] = 0
    flag = rng.random(r) < 0.5
    S["key"] = np.where(flag, S["key"] | FLAG, S["key"])
    return L, S


def split(recs, N):
    k = recs["key"] & ~FLAG
    mask = np.uint64((1 << N) - 1)
    return k & mask, k >> np.uint64(N), recs["re"], recs["im"], ((recs["key"] & FLAG) != 0).astype(np.int32)
