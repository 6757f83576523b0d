"""The greedy refinement's tile-skipping rule (batched_refine_need_kernel), on
the host: where a contender's FP32 value less its error bound is at least the
FP32 curve plus the curve's bound, the FP64 value is at least the FP64 curve,
so min(M64, D64) = M64 and the FP64 tile may be skipped.  Checked on oracle
(FP64) profiles with FP32 stand-ins perturbed by up to the FP32 path's 2e-6
in rho (every cell pushed to the edge of its bound, in random directions), for
every greedy step's contenders; a rule deciding on a tile's mean is caught."""
import numpy as np

import oracle
import synth

DRHO = 2e-6


def value_bound(x, c):
    """Largest change of d = sqrt(2 ell (1 - rho)) at d = x when rho moves by
    c / (2 ell) (the device's value_bound, c = 2.2 ell * 2e-6)."""
    x = np.asarray(x, dtype=np.float64)
    x2 = x * x
    with np.errstate(divide="ignore", invalid="ignore"):
        up = c / (np.sqrt(x2 + c) + x)
        hi = c / (x + np.sqrt(np.maximum(x2 - c, 0.0)))
    return np.where(x2 > c, hi, np.maximum(x, up))


def perturbed(D64, ell, rng):
    """FP32-like values: each cell's rho moved by up to 2e-6, d recomputed."""
    rho = 1.0 - D64 ** 2 / (2.0 * ell)
    rho = rho + rng.uniform(-DRHO, DRHO, size=D64.shape)
    return np.sqrt(2.0 * ell * np.maximum(0.0, 1.0 - rho))


def skip_tiles(row32, M32, W, c, on_average=False):
    """Tiles the rule skips: every position's FP32 value less its bound at least
    the FP32 curve plus its bound.  on_average plants a plausible mistake: the
    test on the tile's mean instead of at every position."""
    b = 1.02 * value_bound(row32, c)
    bm = 1.02 * value_bound(M32, c)
    need = row32 - b < M32 + bm + 1e-5 * (1.0 + M32)
    P = row32.shape[0]
    out = []
    for t in range((P + W - 1) // W):
        sl = slice(t * W, (t + 1) * W)
        if on_average:
            if np.mean(row32[sl] - b[sl]) >= np.mean(M32[sl] + bm[sl]):
                out.append(t)
        elif not need[sl].any():
            out.append(t)
    return out


def test_skipped_tiles_hold_the_fp64_curve():
    s = synth.four_regimes()
    m, ell, k = 128, 64, 13
    D64 = oracle.profiles(s.T, m, ell, k)
    rng = np.random.default_rng(7)
    D32 = perturbed(D64, ell, rng)
    c = 2.2 * ell * DRHO
    W = 64
    chosen, _ = oracle.greedy(D64, 4)
    skipped_any = 0
    for t in range(1, 4):
        M64 = D64[list(chosen[:t])].min(axis=0)
        M32 = D32[list(chosen[:t])].min(axis=0)
        for seg in range(D64.shape[0]):
            if seg in chosen[:t]:
                continue
            for tile in skip_tiles(D32[seg], M32, W, c):
                sl = slice(tile * W, (tile + 1) * W)
                assert np.all(D64[seg, sl] >= M64[sl]), (t, seg, tile)
                skipped_any += 1
    assert skipped_any > 100  # the rule does skip tiles


def test_a_tile_mean_rule_is_caught():
    """Deciding on the tile's mean would skip tiles where the FP64 row dips
    below the FP64 curve at some positions."""
    s = synth.four_regimes()
    m, ell, k = 128, 64, 13
    D64 = oracle.profiles(s.T, m, ell, k)
    c = 2.2 * ell * DRHO
    chosen, _ = oracle.greedy(D64, 2)
    M64 = D64[chosen[0]]
    bad = 0
    for seg in range(D64.shape[0]):
        if seg == chosen[0]:
            continue
        for tile in skip_tiles(D64[seg], M64, 64, c, on_average=True):
            sl = slice(tile * 64, (tile + 1) * 64)
            bad += int(np.any(D64[seg, sl] < M64[sl]))
    assert bad > 0
