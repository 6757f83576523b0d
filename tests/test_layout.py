"""Host logic of the tile-layout choice (no device): the cost model's layouts,
and tuned-table entries, obey the kernel's constraints for every length of the
workloads in both precisions, and a tuned entry that does not fit is ignored."""
import pytest

from paper_2401_13680_b300 import pastila

SMEM = 232448 - 1024  # B300 opt-in shared memory per block, less the headroom for static shared memory


@pytest.mark.parametrize("prec", [pastila.FP32, pastila.FP64])
@pytest.mark.parametrize("n", [4096, 100_000, 1_000_000])
def test_cost_model_layouts_obey_the_kernel_constraints(prec, n):
    pastila.tune_clear()
    for m in list(range(64, 769, 32)) + [8, 24, 50, 100]:
        if m > n:
            continue
        for ell in sorted({m // 2, max(2, m // 8), m}):
            R = m - ell + 1
            lay = pastila.plan_layout(prec, n, m, SMEM, ell=ell)
            assert lay["W"] % 32 == 0 and lay["W"] >= 32
            assert lay["NT"] <= 512 and lay["NT"] % 32 == 0
            assert lay["bytes"] <= SMEM
            assert lay["CS"] in (1, 2, 4) and lay["W"] % (8 * lay["CS"]) == 0
            assert lay["Rh"] == -(-R // lay["CS"])
            assert lay["NG"] * lay["Rg"] >= lay["Rh"] and (lay["NG"] - 1) * lay["Rg"] < lay["Rh"]
            assert lay["NG"] == 1 or lay["Rg"] >= 4
            assert lay["GS"] == 32  # one warp per run of positions


def test_tuned_entries_are_used_when_they_fit():
    pastila.tune_clear()
    try:
        model = pastila.plan_layout(pastila.FP32, 100_000, 256, SMEM)
        pastila.tune_set(pastila.FP32, 256, 128, 26, 320, 2, 32, 2)
        lay = pastila.plan_layout(pastila.FP32, 100_000, 256, SMEM)
        assert (lay["W"], lay["CS"], lay["GS"]) == (320, 2, 32)
        # the same entry does not fit a small budget: the cost model decides
        small = pastila.plan_layout(pastila.FP32, 100_000, 256, 64 * 1024)
        assert small["bytes"] <= 64 * 1024 and (small["W"], small["CS"]) != (320, 2)
        pastila.tune_clear()
        assert pastila.plan_layout(pastila.FP32, 100_000, 256, SMEM) == model
    finally:
        pastila.tune_clear()


def test_no_layout_fits_a_tiny_budget():
    with pytest.raises(pastila.PastilaError, match="does not fit"):
        pastila.plan_layout(pastila.FP32, 100_000, 512, 4096)
