"""Shared-memory index ranges of the profile tile kernel, checked on the host
(no device) for every layout the cost model or the tuned table can give.

The tile geometry (array sizes and offsets in shared memory) is restated here
and pinned to the library's own by the byte count pastila_plan_layout reports.
The index expressions of the rows phase (prefix, chunk and sparse-table
maxima, the exchange between warps, the row-window maxima written into the
owning CTA), of the k-th selection (one run of positions per warp) and the
sizes of the staging copies are then evaluated for every thread, position,
cluster rank, partial last tile and block size a launch can have, and every
index must fall inside its array.  A mistake of the kind this guards against is
planted in the checker itself (a run that applied the column window's slide
at its first position, reading the window entry before it) and must be
caught."""
import numpy as np
import pytest

from paper_2401_13680_b300 import pastila

SMEM = 232448 - 1024  # B300 opt-in shared memory per block, less the static shared memory
V = 4                 # columns per thread, both precisions


def _a16(x):
    return (x + 15) & ~15


def geometry(prec, m, ell, lay):
    """Array sizes (in elements) and the byte count of one tile's shared memory."""
    es = 8 if prec == pastila.FP64 else 4  # working precision and key size alike
    R = m - ell + 1
    W, CS, Rg, NG = lay["W"], lay["CS"], lay["Rg"], lay["NG"]
    Wb = W + R - 1
    NTc = ((Wb + V - 1) // V + 31) // 32 * 32
    NWc = NTc // 32
    Wc = W // CS
    LA = (Wc + V - 1) // V
    RS = (V * LA) | 1
    AE = 16 // es
    RSt = (R + 2 * AE + AE - 1) // AE * AE
    n = dict(AB=R * RS, CB=Wb + 32, PRE=NG * 2 * NTc * V + 16, LV=NG * 2 * 5 * NTc,
             XCH=NG * 4 * NWc, rst=4 * R, row=5 * RSt, left=R, top=NG * NTc * V, Tc=NTc * V + ell + 64,
             Tcl=NTc * V + ell + 64, Ts=m + 2 * AE, Tsl=m + 2 * AE, q=NG * (ell + 1),
             CBp=CS * (Wb + 32) if CS > 1 else 0)
    o = 0
    for k in ("AB", "CB", "PRE", "LV", "XCH", "rst", "row", "left", "top", "Tc", "Tcl", "Ts", "Tsl", "q", "CBp"):
        o = _a16(o + es * n[k])
    return dict(n, R=R, W=W, Wb=Wb, NTc=NTc, NWc=NWc, Wc=Wc, LA=LA, RS=RS, RSt=RSt, AE=AE, es=es,
                CS=CS, Rg=Rg, NG=NG, GS=lay["GS"], NT=lay["NT"], ell=ell, m=m, bytes=o)


def _tdiv(a, b):
    """C integer division (towards zero) and remainder, elementwise."""
    q = np.trunc(a / b).astype(np.int64)
    return q, a - q * b


def selection_reads(G, BD, crank, Wp, slide_at_start=False):
    """(AB index range, CB index range) over every read of the selection phase of
    CTA crank of a tile with Wp positions, launched with BD threads: one run of
    consecutive positions per warp; lane l reads rows l + 32 j of each position's
    AB column and its window entries p + l + 32 j, and every position after a
    run's first also reads the window entries that leave (p - 1) and enter
    (p + R - 1).  slide_at_start plants the mistake of sliding the window at a
    run's first position as well."""
    R, Wc, LA, RS = G["R"], G["Wc"], G["LA"], G["RS"]
    pofs = crank * Wc
    Wn = max(0, min(Wp - pofs, Wc))
    nwarps = BD >> 5
    PW = (Wn + nwarps - 1) // nwarps
    if PW == 0:
        return None, None
    ab_l, cb_l = [], []
    for w in range(nwarps):
        pb = w * PW
        npos = 0 if pb >= Wn else min(PW, Wn - pb)
        if npos == 0:
            continue
        p = pofs + pb + np.arange(npos)
        q, r = _tdiv(p - pofs, V)
        cp = r * LA + q  # AB column of each position; rows at multiples of RS
        ab_l += [cp.min(), (R - 1) * RS + cp.max()]
        cb_l += [p.min(), p.max() + R - 1]
        slid = p if slide_at_start else p[1:]
        if slid.size:
            cb_l += [slid.min() - 1]
    ab, cb = np.array(ab_l), np.array(cb_l)
    return (int(np.min(ab)), int(np.max(ab))), (int(np.min(cb)), int(np.max(cb)))


def _assert_union(pieces, lo, hi):
    """The column (or chunk) ranges cover lo .. hi exactly: nothing outside, no
    gap (overlaps are harmless for a maximum)."""
    pieces = sorted(pieces)
    assert all(lo <= a_ <= b_ <= hi for a_, b_ in pieces), (pieces, lo, hi)
    assert pieces[0][0] == lo, (pieces, lo)
    reach = pieces[0][1]
    for a_, b_ in pieces[1:]:
        assert a_ <= reach + 1, (pieces, lo, hi)
        reach = max(reach, b_)
    assert reach == hi, (pieces, hi)


def rows_phase_check(G, Wp):
    """Every shared-memory index of the rows phase of a tile with Wp positions
    (per row group and parity: the prefix maxima within each chunk PRE, stored
    by column; the sparse tables LV [NTc][5] of the chunk maxima (level 0) and
    of 2, 4, 8, 16 consecutive chunks; the warp exchange XCH [NWc][parity][2]; the row
    statistics [R][4]; the row-window maxima written into the owning CTA's AB)
    lies inside its array, each sparse-table read spans chunks of one warp, and
    the pieces of every owned position's window (own suffix, whole chunks in
    between, the far chunk's prefix) cover exactly its R columns."""
    R, V_, NTc, NWc = G["R"], V, G["NTc"], G["NWc"]
    RS, LA, Wc, CS = G["RS"], G["LA"], G["Wc"], G["CS"]
    per_par_pre = NTc * V_
    q0 = (R - 1) // V_
    rr = (R - 1) - q0 * V_
    small_R = R - 1 < V_
    t = np.arange(NTc)
    xb = t * V_
    # writes of every active thread (all column threads take part in every row step)
    assert per_par_pre + xb.max() + V_ - 1 < G["PRE"] // G["NG"]  # PRE, parity 1
    assert 5 * NTc + t.max() * 5 + 4 < 2 * 5 * NTc                # LV, parity 1, level 4
    assert (NWc - 1) * 4 + 1 * 2 + 1 < 4 * NWc                    # XCH, last warp, parity 1
    assert 4 * (R - 1) + 3 < G["rst"]
    owners = xb < Wp
    for tt in (int(x) for x in t[owners]):
        x0 = tt * V_
        # every far read (all V of the thread, owned or not) stays inside PRE
        assert per_par_pre + x0 + V_ - 1 + R - 1 < G["PRE"] // G["NG"]
        # window pieces, as column ranges relative to the tile
        for i in range(V_):
            if x0 + i >= Wp:
                continue
            e = i + R - 1
            oi, si = e // V_, e % V_
            assert x0 + e == (tt + oi) * V_ + si and tt + oi <= NTc - 1  # PRE column of the far prefix
            lo, hi = x0 + i, x0 + i + R - 1
            if small_R and e < V_:
                cover = [(lo, hi)]                       # inside this chunk
            else:
                cover = [(x0 + i, x0 + V_ - 1)]          # own suffix
                if not small_R and q0 >= 2:
                    cover.append(((tt + 1) * V_, (tt + q0) * V_ - 1))  # whole chunks t+1 .. t+q0-1
                if not small_R and i + rr >= V_:
                    assert oi > q0
                    cover.append(((tt + q0) * V_, (tt + q0 + 1) * V_ - 1))  # chunk t+q0
                cover.append(((tt + oi) * V_, (tt + oi) * V_ + si))  # far chunk's prefix
            _assert_union(cover, lo, hi)
        if not small_R and rr > 0:
            assert (tt + q0) * 5 < 5 * NTc               # LV level 0 at t + q0
        if not small_R and q0 >= 2:
            a_, z_ = tt + 1, tt + q0 - 1
            wa, wz = a_ >> 5, z_ >> 5
            spans = [(a_, z_)] if wa == wz else [(a_, wa * 32 + 31), (wz * 32, z_)]
            pieces = []
            for x, y in spans:
                k = min(int(y - x + 1).bit_length() - 1, 4)
                w = 1 << k
                for s0 in (x, y - w + 1):
                    assert s0 >> 5 == (s0 + w - 1) >> 5 and 0 <= s0 and s0 + w - 1 < NTc
                    assert s0 * 5 + k < 5 * NTc
                    pieces.append((s0, s0 + w - 1))
            for wv in range(wa + 1, wz):
                assert (wv * 32 + 16) * 5 + 4 < 5 * NTc
                pieces += [(wv * 32, wv * 32 + 15), (wv * 32 + 16, wv * 32 + 31)]
            _assert_union(pieces, a_, z_)
            if rr == 0 and 2 <= q0 <= 65:
                # the fast row steps read one whole warp at most, and only past
                # q0 = 33; no read reaches a chunk past the window of the tile
                whole = max(0, wz - wa - 1)
                assert whole <= 1 and (whole == 0 or q0 > 33)
                if Wp % V_ == 0:
                    assert z_ <= (Wp + R - 1) // V_ - 1
        # the row-window maxima of this thread's positions, into the owner's AB
        owner = x0 // Wc if CS > 1 else 0
        tofs = owner * (Wc // V_) if CS > 1 else 0
        for i in range(V_):
            if x0 + i < Wp:
                assert owner == (x0 + i) // Wc or CS == 1
                idx = (R - 1) * RS + (tt - tofs) + i * LA
                assert 0 <= tt - tofs and idx < R * RS


def check_layout(prec, m, ell, lay):
    G = geometry(prec, m, ell, lay)
    assert G["bytes"] == lay["bytes"], (m, ell, lay, G["bytes"])  # the restatement is the library's geometry
    assert G["Wc"] % V == 0  # a thread's V positions share one owner CTA
    R, AE = G["R"], G["AE"]
    # the rows phase's indices do not depend on the CTA's rank, and a partial
    # tile owns a subset of a full tile's positions
    rows_phase_check(G, G["W"])
    for BD in sorted({G["NT"], min(512, G["NT"] + 32), 512}):
        if BD < G["NT"]:
            continue
        for crank in range(G["CS"]):
            for Wp in sorted({G["W"], G["W"] - 1, G["W"] // 2 + 3, G["Wc"] + 1, 1} - {0}):
                if not 1 <= Wp <= G["W"]:
                    continue
                abr, cbr = selection_reads(G, BD, crank, Wp)
                if abr is None:
                    continue
                assert 0 <= abr[0] and abr[1] < G["AB"], (m, ell, lay, BD, crank, Wp, abr, G["AB"])
                assert 0 <= cbr[0] and cbr[1] < Wp + R - 1 + 32 <= G["CB"], (m, ell, lay, BD, crank, Wp, cbr)
                # staging copies of this tile: whole 16-byte units from a 16-byte boundary
                nTc = Wp + R - 1 + ell - 1
                assert (nTc + AE - 1) // AE * AE <= G["Tc"]
                for os in range(AE):
                    assert (os + m + AE - 1) // AE * AE <= G["Ts"]
                    assert (os + R + AE - 1) // AE * AE <= G["RSt"]
    # the seeds' sliding reads (9-column blocks) stay inside the staged window
    J = 9
    nblk = (G["NTc"] * V + J - 1) // J
    assert (nblk - 1) * J + ell - 1 + J < G["Tc"]
    # the group seeds take one block per thread on the first tA threads (whole
    # warps); where a warp is left over, the rest form the head sums, arrive on
    # barrier 1 (count: every thread of the CTA, a multiple of 32) and compute
    # the left edge, while the group seeds wait there once each
    tA = (G["NG"] * nblk + 31) // 32 * 32
    for BD in sorted({G["NT"], min(512, G["NT"] + 32), 512}):
        if BD < G["NT"]:
            continue
        assert BD % 32 == 0 and tA >= G["NG"] * nblk
        if tA + 32 <= BD:
            warps_b = (BD - tA) // 32
            assert warps_b >= 1 and tA % 32 == 0
            # every group's head sum has a warp (warp w takes groups w, w + warps_b, ...)
            assert all(any(gg % warps_b == w for w in range(warps_b)) for gg in range(G["NG"]))
    # row-window maxima of owned positions end inside the chunk prefix arrays
    assert G["W"] - 1 + R - 1 <= G["NTc"] * V - 1


def _cases():
    ms = [8, 24, 50, 100] + list(range(64, 769, 32))
    for prec in (pastila.FP32, pastila.FP64):
        for n in (4096, 100_000, 1_000_000):
            for m in ms:
                if m > n:
                    continue
                for ell in sorted({m // 2, max(2, m // 8), m}):
                    yield prec, n, m, ell


@pytest.mark.parametrize("prec", [pastila.FP32, pastila.FP64])
def test_cost_model_layouts_stay_in_bounds(prec):
    pastila.tune_clear()
    count = 0
    for p, n, m, ell in _cases():
        if p != prec:
            continue
        check_layout(prec, m, ell, pastila.plan_layout(prec, n, m, SMEM, ell=ell))
        count += 1
    assert count > 100


@pytest.mark.parametrize("CS", [1, 2, 4])
def test_tuned_layouts_stay_in_bounds(CS):
    """Layouts forced through the tuned table: every width and row-group count
    the tuner can choose, with one, two and four CTAs per tile."""
    pastila.tune_clear()
    checked = 0
    try:
        for m in (64, 128, 256, 512, 640):
            ell = m // 2
            k = (m + 9) // 10
            R = m - ell + 1
            for W in range(32 * CS, 1025, 32 * CS):
                for NGw in (1, 2, 3, 4):
                    pastila.tune_set(pastila.FP32, m, ell, k, W, NGw, 32, CS)
                    lay = pastila.plan_layout(pastila.FP32, 1_000_000, m, SMEM, ell=ell, k=k)
                    if (lay["W"], lay["CS"]) != (W, CS):
                        continue  # does not fit: the cost model decides instead
                    check_layout(pastila.FP32, m, ell, lay)
                    checked += 1
    finally:
        pastila.tune_clear()
    assert checked > 20


def test_checker_catches_a_window_slide_at_a_run_start():
    """A run that slid the column window at its first position would read the
    window entry before the first position of the tile (index -1 of CB)."""
    pastila.tune_clear()
    m, ell = 512, 256
    try:
        pastila.tune_set(pastila.FP32, m, ell, 52, 256, 4, 32, 2)
        lay = pastila.plan_layout(pastila.FP32, 100_000, m, SMEM, ell=ell, k=52)
    finally:
        pastila.tune_clear()
    G = geometry(pastila.FP32, m, ell, lay)
    assert G["CS"] == 2
    Wp = G["W"] - 5  # a partial tile
    _, good = selection_reads(G, G["NT"], 0, Wp)
    _, bad = selection_reads(G, G["NT"], 0, Wp, slide_at_start=True)
    assert good[0] >= 0
    assert bad[0] < 0


def test_cost_model_counts_the_columns_the_threads_compute():
    """The layout model pays the rows on the NTc V columns the column threads
    compute (W + R - 1 rounded up to whole warps), so its choice for every length
    of the benchmark sweep computes few columns past W + R - 1."""
    pastila.tune_clear()
    for m in range(64, 513, 32):
        ell = m // 2
        lay = pastila.plan_layout(pastila.FP32, 100_000, m, SMEM, ell=ell)
        G = geometry(pastila.FP32, m, ell, lay)
        Wb = G["W"] + G["R"] - 1
        assert G["NTc"] * V <= 1.1 * Wb, (m, lay, G["NTc"] * V, Wb)
