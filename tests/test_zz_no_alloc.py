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

import synth

pytestmark = pytest.mark.gpu


def test_greedy_noalloc_matches_snippets(lib):
    import torch
    from paper_2401_13680_b300 import pastila

    s = synth.four_regimes()
    dev = torch.device("cuda", 0)
    K = 4
    with pastila.Series(s.T, precision=pastila.FP32) as h:
        # two calls in a row, with different sizes, through the one shared scratch array
        for m in (128, 96):
            S, P = h.n // m, h.n - m + 1
            D = torch.empty((S, P), dtype=torch.float32, device=dev)
            h.profiles_device(m, D.data_ptr())
            torch.cuda.synchronize()
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
