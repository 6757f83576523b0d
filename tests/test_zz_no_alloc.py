"""The allocation-free greedy search (pastila_greedy_noalloc) against the
regular snippet entry point.

pastila_greedy_noalloc exists for callers that cannot allocate device memory
themselves, for instance code whose device memory is handed out by another
allocator or that must not allocate inside its hot loop: it takes the profile
set and the output buffers from the caller and keeps its own working storage
in a fixed array inside the library.  This file is collected last so that a
run stopping at its first failure has run every other test first."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def test_greedy_noalloc_matches_snippets(lib):
    import torch
    from paper_2401_13680_b300 import pastila

    s = synth.four_regimes()
    dev = torch.device("cuda", 0)
    K = 4
    with pastila.Series(s.T, precision=pastila.FP32) as h:
        # the allocation-free search decides every step on FP32 areas, as
        # pastila_snippets does with the FP64 re-evaluation of near-ties off
        h.set_fp64_ties(False)
        # two calls in a row, with different sizes, through the one shared scratch array
        for m in (128, 96):
            S, P = h.n // m, h.n - m + 1
            D = torch.empty((S, P), dtype=torch.float32, device=dev)
            h.profiles_device(m, D.data_ptr())
            torch.cuda.synchronize()
            h.stage_status()  # the enqueue-only call's staging waits completed
            chosen = torch.full((K,), -1, dtype=torch.int32, device=dev)
            area = torch.zeros(K, dtype=torch.float64, device=dev)
            pastila.greedy_noalloc(D.data_ptr(), S, P, K, chosen.data_ptr(), area.data_ptr(),
                                   torch.cuda.current_stream().cuda_stream)
            torch.cuda.synchronize()
            recs, _, _ = h.snippets(m, K)
            by_step = sorted(recs, key=lambda r: r[1])
            assert chosen.cpu().tolist() == [r[0] for r in by_step]
            np.testing.assert_allclose(area.cpu().numpy(), [r[3] for r in by_step], rtol=1e-12)


def test_greedy_noalloc_rejects_sizes_beyond_its_scratch(lib):
    from paper_2401_13680_b300 import pastila

    with pytest.raises(pastila.PastilaError, match="exceeds"):
        pastila.greedy_noalloc(1 << 20, 16385, 1000, 2, 1 << 20, 1 << 20)
    with pytest.raises(pastila.PastilaError, match="exceeds"):
        pastila.greedy_noalloc(1 << 20, 100, (1 << 20) + 1, 2, 1 << 20, 1 << 20)
    with pytest.raises(pastila.PastilaError, match="K = 0"):
        pastila.greedy_noalloc(1 << 20, 100, 1000, 0, 1 << 20, 1 << 20)


def _exact_rows(rng, S, P, scale_exp, lo_bits, hi_bits, zeros):
    """S x P binary32 values k * 2^scale_exp with integers k drawn log-uniformly
    between 2^lo_bits and 2^hi_bits (every FP64 sum of up to P of them is then
    exact), a share of exact zeros and one negative zero."""
    k = np.floor(np.exp2(rng.uniform(lo_bits, hi_bits, size=(S, P))))
    D = np.ldexp(np.maximum(k, 1.0), scale_exp)
    D[rng.random((S, P)) < zeros] = 0.0
    D = D.astype(np.float32)
    D[0, 1] = -0.0
    return D


@pytest.mark.parametrize("case", ["subnormal", "ordinary", "near_max"])
def test_greedy_area_sums_exact(lib, case):
    """The FP32 area sums widen every binary32 value to binary64 exactly.  On
    profile sets whose every sum is exact in FP64 (integer multiples of one
    power of two, totals below 2^53 of it), the areas after each step equal
    the oracle's to the last bit, and so do the chosen segments: subnormal and
    smallest normal values (multiples of 2^-149 below 2^-110), ordinary
    magnitudes, and values near the binary32 maximum."""
    import torch
    from paper_2401_13680_b300 import pastila

    rng = np.random.default_rng({"subnormal": 11, "ordinary": 12, "near_max": 13}[case])
    S, P = 6, 5003  # several strides of the 4-way unrolled loop and a ragged tail
    if case == "subnormal":
        D = _exact_rows(rng, S, P, -149, 0, 39, 0.05)   # below 2^-110: subnormals and small normals
    elif case == "ordinary":
        D = _exact_rows(rng, S, P, -10, 0, 20, 0.05)    # below 2^10
    else:
        D = _exact_rows(rng, S, P, 104, 20, 24, 0.05)   # up to 2^128 (binary32 maximum)
    if case == "subnormal":  # both subnormal and normal binary32 values present
        nz = np.abs(D[D != 0])
        assert (nz < np.float32(2.0 ** -126)).mean() > 0.3 and (nz >= np.float32(2.0 ** -126)).mean() > 0.3
    K = S
    ref_chosen, ref_area = oracle.greedy(D.astype(np.float64), K)
    dev = torch.device("cuda", 0)
    Dd = torch.from_numpy(D).to(dev)
    chosen = torch.full((K,), -1, dtype=torch.int32, device=dev)
    area = torch.zeros(K, dtype=torch.float64, device=dev)
    pastila.greedy_noalloc(Dd.data_ptr(), S, P, K, chosen.data_ptr(), area.data_ptr(),
                           torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert chosen.cpu().tolist() == ref_chosen.tolist()
    np.testing.assert_array_equal(area.cpu().numpy(), ref_area)
