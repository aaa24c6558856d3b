"""Checks that pin the CPU oracle to the paper and to mathematics, not to itself.

Each ``pin_*`` function takes an ``oracle.Oracle`` and returns a list of
``(name, ok, detail)``.  ``test_oracle_pins.py`` requires every check to pass
on the real oracle; ``test_oracle_mutants.py`` builds the oracle with one
planted mistake at a time and requires at least one check to fail for each.

What each pin leans on (none of it re-types the oracle's own formulas):
  * exact rational arithmetic (``fractions``) for the Eq. 3 fold and the
    magnitude binning on small inputs;
  * the plain epoch fold (Pdot = 0) computed with numpy;
  * the Eq. 6 dephasing law (phase shift 1/2 |Pdot| t^2 / P^2);
  * the chain rule H(M|Phi) = H(M, Phi) - H(Phi) with scipy's Shannon entropy,
    and its special cases (one phase bin: the magnitude histogram's entropy;
    one magnitude bin or one point per phase bin: zero);
  * invariants of Eq. 4 (bounds, permutation invariance);
  * the paper's worked example (Fig. 2: P = 7 min, Pdot = -2.14e-11, ten years
    of weekly visits) and on-grid recovery of injected signals;
  * numpy's median and standard deviation for the per-filter normalisation of
    multi-filter input, and a closed form for a calibrated copy of a filter.
"""
from __future__ import annotations

import json
import math
import os
from fractions import Fraction

import numpy as np
from scipy.stats import entropy as shannon

import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return json.load(fh)


# ----------------------------------------------------------------- exact fold

def _dyadic(rng, lo, hi, bits=20):
    """A random float64 in [lo, hi) with at most `bits` fractional binary digits
    below its leading scale, so that it converts to Fraction exactly."""
    x = rng.uniform(lo, hi)
    e = math.frexp(x)[1]
    q = 2.0 ** (e - bits)
    return float(round(x / q) * q)


def exact_phase_scaled(tau, period, pdot, n_phase):
    """frac(tau/P - 1/2 Pdot tau^2 / P^2) * n_phase in exact rational arithmetic."""
    t = Fraction(tau)
    p = Fraction(period)
    d = Fraction(pdot)
    x = t / p - Fraction(1, 2) * d * t * t / (p * p)
    fr = x - math.floor(x)
    return fr * n_phase


def pin_fold_exact_rational(orc):
    """Eq. 3 against exact arithmetic: for points not within 1e-7 (in units of
    phase bins) of an edge, the oracle's phase bin is the exact one."""
    rng = np.random.default_rng(7)
    out = []
    bad = 0
    checked = 0
    for trial in range(400):
        n_phase = int(rng.integers(2, 60))
        period = _dyadic(rng, 60.0, 90000.0)
        pdot = 0.0 if trial % 4 == 0 else _dyadic(rng, -1e-10, 1e-10, bits=30)
        t0 = _dyadic(rng, -1e7, 1e7)
        f, a = orc.trial_constants(period, pdot)
        for _ in range(8):
            t = _dyadic(rng, 0.0, 3.2e8)
            tau = t - t0
            ex = exact_phase_scaled(Fraction(t) - Fraction(t0), period, pdot, n_phase)
            j_ex = math.floor(ex)
            dist = min(ex - j_ex, j_ex + 1 - ex)
            if dist < Fraction(1, 10**7):
                continue
            j, _ = orc.phase_bin(tau, f, a, n_phase)
            # the oracle folds tau - t0 itself in its batch path; here tau is exact
            checked += 1
            if j != j_ex:
                bad += 1
    out.append(("fold matches exact rational phase bin", bad == 0 and checked > 2000,
                f"{bad} mismatches of {checked}"))

    # the batch path's epoch handling: a whole cell with t0 != 0 against exact bins
    bad_cells = 0
    cells = 0
    worst_dmin = 0.0
    for trial in range(40):
        n_phase = int(rng.integers(2, 30))
        n_mag = int(rng.integers(1, 12))
        period = _dyadic(rng, 100.0, 5000.0)
        pdot = _dyadic(rng, -1e-10, 1e-10, bits=30)
        t0 = _dyadic(rng, -1e8, 1e8)
        t = np.array([_dyadic(rng, 0.0, 1e8) for _ in range(8)])
        m = np.array([_dyadic(rng, 14.0, 16.0) for _ in range(8)])
        h, counts, dmin = orc.cell(t, m, t0, period, pdot, n_phase, n_mag)
        exact_counts = exact_cell_counts(t, m, t0, period, pdot, n_phase, n_mag)
        if exact_counts is None:
            continue
        cells += 1
        if not np.array_equal(counts, exact_counts):
            bad_cells += 1
        # the edge distance the parity tests use: min over points of the exact phase's
        # distance from a bin edge, in cycles (the fold's own rounding is ~1e-9 here)
        ex = [exact_phase_scaled(Fraction(float(tk)) - Fraction(t0), period, pdot, n_phase)
              for tk in t]
        want = min(min(e - math.floor(e), math.floor(e) + 1 - e) for e in ex) / n_phase
        worst_dmin = max(worst_dmin, abs(dmin - float(want)))
    out.append(("cell counts with epoch t0 match exact arithmetic",
                bad_cells == 0 and cells >= 20, f"{bad_cells} of {cells} cells differ"))
    out.append(("edge distance dmin matches exact arithmetic (cycles)", worst_dmin < 1e-8,
                f"worst {worst_dmin:.3g}"))
    return out


def exact_mag_bins(m, n_mag):
    fm = [Fraction(float(v)) for v in m]
    mn, mx = min(fm), max(fm)
    if mx == mn:
        return [0] * len(fm), [Fraction(1)] * len(fm)
    bins, dists = [], []
    for v in fm:
        y = (v - mn) / (mx - mn) * n_mag
        i = min(math.floor(y), n_mag - 1)
        bins.append(i)
        # the extremes are exact in floating point too (0 and the clamped top)
        exact_end = v == mx or v == mn
        dists.append(Fraction(1) if exact_end else min(y - math.floor(y), math.floor(y) + 1 - y))
    return bins, dists


def exact_cell_counts(t, m, t0, period, pdot, n_phase, n_mag, margin=Fraction(1, 10**7)):
    """Counts from exact arithmetic, or None when a point sits within `margin`
    of a phase or magnitude edge (where float rounding may legitimately differ)."""
    bins, mdist = exact_mag_bins(m, n_mag)
    counts = np.zeros((n_mag, n_phase), dtype=np.int64)
    for tk, ik, dk in zip(t, bins, mdist):
        if dk < margin:
            return None
        ex = exact_phase_scaled(Fraction(float(tk)) - Fraction(float(t0)), period, pdot, n_phase)
        j = math.floor(ex)
        if min(ex - j, j + 1 - ex) < margin:
            return None
        counts[ik, j] += 1
    return counts


def pin_fold_edges(orc):
    """Bin edges: a phase exactly on an edge belongs to the upper bin (floor), the
    double just below it to the lower bin, and phi*n_phase rounding up to n_phase
    (a tiny negative x, whose x - floor(x) rounds to 1.0) is clamped into the
    last bin."""
    out = []
    ok = True
    for n_phase in (2, 4, 8, 16, 32):
        for j in range(n_phase):
            tau = 12345.0 + j / n_phase  # exact in binary
            jj, _ = orc.phase_bin(tau, 1.0, 0.0, n_phase)
            ok &= jj == j
            below = math.nextafter(tau, -math.inf)
            jb, _ = orc.phase_bin(below, 1.0, 0.0, n_phase)
            ok &= jb == (j - 1) % n_phase
    out.append(("edges: floor puts an on-edge phase in the upper bin", ok, ""))
    # a tiny negative x: x - floor(x) = x + 1 rounds to exactly 1.0
    j, y = orc.phase_bin(-(2.0 ** -60), 1.0, 0.0, 5)
    out.append(("phase rounding up to a full cycle is clamped into the last bin",
                j == 4 and y == 5.0, f"j={j} y={y}"))
    return out


def pin_pdot_zero_plain_fold(orc):
    """With Pdot = 0, Eq. 3 is the plain epoch fold frac(tau/P) (computed here
    with numpy as frac(tau * (1/P)))."""
    rng = np.random.default_rng(11)
    bad = 0
    for _ in range(2000):
        period = rng.uniform(60.0, 1e5)
        tau = rng.uniform(-1e8, 3e8)
        n_phase = int(rng.integers(1, 100))
        f, a = orc.trial_constants(period, 0.0)
        j, y = orc.phase_bin(tau, f, a, n_phase)
        x = np.float64(tau) * np.float64(1.0 / period)
        ph = x - np.floor(x)
        yy = ph * n_phase
        jj = min(int(np.floor(yy)), n_phase - 1)
        if j != jj or y != yy:
            bad += 1
    return [("Pdot = 0 reduces bit-exactly to the plain fold", bad == 0, f"{bad} differ")]


def pin_eq6_dephasing(orc):
    """Eq. 6: including Pdot shifts the folded phase by 1/2 |Pdot| t^2 / P^2
    (advanced for Pdot < 0).  Checked on frac(x) with one phase bin, mod 1."""
    rng = np.random.default_rng(13)
    worst = 0.0
    for _ in range(2000):
        period = rng.uniform(120.0, 4000.0)
        pdot = -(10.0 ** rng.uniform(-13, -10))
        tau = rng.uniform(0.0, 3.2e8)
        f0, a0 = orc.trial_constants(period, 0.0)
        f1, a1 = orc.trial_constants(period, pdot)
        _, y0 = orc.phase_bin(tau, f0, a0, 1)
        _, y1 = orc.phase_bin(tau, f1, a1, 1)
        expect = 0.5 * abs(pdot) * tau * tau / (period * period)
        d = (y1 - y0 - expect) % 1.0
        d = min(d, 1.0 - d)
        # rounding of x (|x| up to ~3e6 cycles) is ~5e-10; allow 1e-6
        worst = max(worst, d)
    return [("Eq. 6 dephasing 1/2 |Pdot| t^2/P^2 for Pdot < 0", worst < 1e-6,
             f"worst {worst:.3g} cycles")]


def pin_mag_bins(orc):
    """Min-max magnitude binning against exact arithmetic, including values exactly
    on edges and the maximum (clamped into the last bin)."""
    out = []
    rng = np.random.default_rng(17)
    ok = True
    for n_mag in (1, 2, 3, 5, 10, 16, 255):
        # edges: mn + k/n_mag * (mx - mn) with a power-of-two range
        mn, span = 14.0, 2.0
        vals = [mn + span * k / n_mag for k in range(n_mag)] + [mn + span]
        vals = np.array(vals)
        got = orc.mag_bins(vals, n_mag)
        exp, _ = exact_mag_bins(vals, n_mag)
        # exact-on-edge values where float division is exact when n_mag is a power of 2
        if n_mag & (n_mag - 1) == 0:
            ok &= list(got) == exp
        ok &= got[-1] == n_mag - 1 and got[0] == 0
    out.append(("magnitude bins: edges and maximum", ok, ""))
    bad = 0
    for _ in range(300):
        n_mag = int(rng.integers(1, 40))
        m = np.array([_dyadic(rng, 10.0, 20.0) for _ in range(int(rng.integers(2, 30)))])
        got = orc.mag_bins(m, n_mag)
        exp, dist = exact_mag_bins(m, n_mag)
        for g, e, d in zip(got, exp, dist):
            if d > Fraction(1, 10**9) and g != e:
                bad += 1
    out.append(("magnitude bins match exact arithmetic", bad == 0, f"{bad} differ"))
    const = orc.mag_bins(np.full(7, 15.25), 10)
    out.append(("all-equal magnitudes fall in bin 0", bool(np.all(const == 0)), ""))
    return out


def chain_rule_entropy(counts):
    """H(M | Phi) = H(M, Phi) - H(Phi), each a Shannon entropy (nats, scipy)."""
    c = np.asarray(counts, dtype=np.float64)
    if c.sum() == 0:
        return 0.0
    joint = shannon(c.ravel())
    marg = shannon(c.sum(axis=0))
    return float(joint - marg)


def pin_entropy_chain_rule(orc):
    """Eq. 4 equals the chain-rule conditional entropy H(M, Phi) - H(Phi)."""
    rng = np.random.default_rng(19)
    worst = 0.0
    for _ in range(500):
        n_mag = int(rng.integers(1, 20))
        n_phase = int(rng.integers(1, 60))
        lam = rng.uniform(0.05, 30.0)
        counts = rng.poisson(lam, size=(n_mag, n_phase))
        counts[rng.random(size=counts.shape) < 0.3] = 0
        if counts.sum() == 0:
            counts[0, 0] = 1
        h = orc.entropy(counts)
        worst = max(worst, abs(h - chain_rule_entropy(counts)))
    return [("Eq. 4 equals H(M,Phi) - H(Phi)", worst < 1e-12, f"worst {worst:.3g}")]


def pin_entropy_special_cases(orc):
    rng = np.random.default_rng(23)
    out = []
    worst = 0.0
    for _ in range(200):
        n_mag = int(rng.integers(1, 20))
        counts = rng.integers(0, 50, size=(n_mag, 1))
        if counts.sum() == 0:
            counts[0, 0] = 3
        h = orc.entropy(counts)
        worst = max(worst, abs(h - shannon(counts[:, 0].astype(float))))
    out.append(("one phase bin: Shannon entropy of the magnitude histogram",
                worst < 1e-12, f"worst {worst:.3g}"))
    z1 = orc.entropy(rng.integers(0, 9, size=(1, 17)) + 1)
    out.append(("one magnitude bin: H = 0", abs(z1) < 1e-15, f"{z1}"))
    own = np.zeros((6, 40), dtype=np.int64)
    for k, i in enumerate(rng.integers(0, 6, size=40)):
        own[i, k] = 1
    z2 = orc.entropy(own)
    out.append(("one point per phase bin: H = 0", abs(z2) < 1e-15, f"{z2}"))
    return out


def pin_entropy_bounds_and_invariance(orc):
    """0 <= H <= min(ln n_mag, ln N); permuting points leaves counts and H alone;
    a constant light curve has H = 0 at every trial."""
    rng = np.random.default_rng(29)
    out = []
    ok = True
    perm_ok = True
    for _ in range(60):
        n = int(rng.integers(1, 200))
        n_mag = int(rng.integers(1, 16))
        n_phase = int(rng.integers(1, 40))
        t = np.sort(rng.uniform(0, 1e8, size=n))
        m = rng.normal(15, 0.3, size=n)
        period = rng.uniform(200, 5000)
        pdot = -rng.uniform(0, 1e-10)
        h, counts, _ = orc.cell(t, m, 0.0, period, pdot, n_phase, n_mag)
        ok &= -1e-15 <= h <= min(math.log(n_mag), math.log(n)) + 1e-12
        ok &= int(counts.sum()) == n
        perm = rng.permutation(n)
        h2, counts2, _ = orc.cell(t[perm], m[perm], 0.0, period, pdot, n_phase, n_mag)
        perm_ok &= np.array_equal(counts, counts2) and abs(h - h2) < 1e-13
    out.append(("0 <= H <= min(ln n_mag, ln N) and counts sum to N", ok, ""))
    out.append(("point order does not matter", perm_ok, ""))
    t = np.sort(rng.uniform(0, 1e8, size=50))
    hs = [orc.cell(t, np.full(50, 15.0), 0.0, p, 0.0, 15, 10)[0] for p in (300.0, 1234.5)]
    out.append(("constant light curve: H = 0", max(abs(x) for x in hs) == 0.0, str(hs)))
    return out


def pin_brute_force_tiny(orc):
    """Whole cells on 8-point inputs: exact-arithmetic counts fed to the chain-rule
    entropy give the oracle's H."""
    rng = np.random.default_rng(31)
    worst = 0.0
    done = 0
    for _ in range(300):
        n_phase = int(rng.integers(1, 12))
        n_mag = int(rng.integers(1, 8))
        period = _dyadic(rng, 100.0, 3000.0)
        pdot = _dyadic(rng, -1e-10, 0.0, bits=30)
        t = np.array([_dyadic(rng, 0.0, 1e8) for _ in range(8)])
        m = np.array([_dyadic(rng, 14.0, 16.0) for _ in range(8)])
        ex = exact_cell_counts(t, m, 0.0, period, pdot, n_phase, n_mag)
        if ex is None:
            continue
        h, _, _ = orc.cell(t, m, 0.0, period, pdot, n_phase, n_mag)
        worst = max(worst, abs(h - chain_rule_entropy(ex)))
        done += 1
    return [("8-point brute force (exact fold + chain rule) gives H", worst < 1e-12 and done > 100,
             f"worst {worst:.3g} over {done}")]


def pin_paper_worked_example(orc):
    """Fig. 2 (Sec. 2.3): an eclipsing binary at P = 7 min, Pdot = -2.14e-11 s/s,
    observed weekly for ten years, folds coherently only with its Pdot.  The
    dephasing at Pdot = 0 is 1/2 |Pdot| T^2 / P^2 (Eq. 6) cycles."""
    g = _golden("paper_numbers.json")["fig2_example"]
    period = g["period_min"] * 60.0
    pdot = g["pdot"]
    years = g["baseline_years"]
    t_end = years * 365.25 * 86400.0
    deph = 0.5 * abs(pdot) * t_end ** 2 / period ** 2
    out = [("Fig. 2 example dephases by the Eq. 6 amount",
            abs(deph - g["dephasing_cycles_eq6"]) < 0.01, f"{deph:.3f} cycles")]
    rng = np.random.default_rng(37)
    n = int(years * 365.25 / g["cadence_days"])
    t = np.sort(np.arange(n) * g["cadence_days"] * 86400.0 + rng.normal(0, 3600.0, size=n))
    t -= t[0]
    cyc = synth.lightcurves.chirp_cycles(t, period, pdot)
    m = 16.0 + synth.lightcurves.eclipse_signal(cyc, 0.6, 0.05, 0.3) + rng.normal(0, 0.02, n)
    h_true, _, _ = orc.cell(t, m, 0.0, period, pdot, 15, 10)
    h_zero, _, _ = orc.cell(t, m, 0.0, period, 0.0, 15, 10)
    out.append(("Fig. 2 example: H(P, Pdot) far below H(P, 0)", h_true + 0.3 < h_zero,
                f"H(Pdot)={h_true:.4f} H(0)={h_zero:.4f}"))
    return out


def pin_recovery(orc):
    """Noiseless signals injected on grid cells: the grid minimum's tie-set contains
    the injected cell (Sec. 2.3: the lowest CE marks the most likely parameters)."""
    out = []
    # P-only: narrow period band (no harmonic of P0 inside it), 3-yr nightly cadence
    ok = True
    for seed in range(6):
        rng = np.random.default_rng(100 + seed)
        p0 = float(np.exp(rng.uniform(np.log(300), np.log(20000))))
        periods = synth.log_periods(p0 * 0.8, p0 * 1.25, 301)
        batch, pi, qi = synth.make_onegrid_injection(200 + seed, 2, 300, periods, [0.0],
                                                     kind="eclipse" if seed % 2 else "sine")
        grid = orc.ce_grid(batch.times, batch.mags, batch.offsets, batch.periods, batch.pdots,
                           15, 10)
        for c in range(batch.n_curves):
            g = grid[c].ravel()
            ties = np.flatnonzero(g <= g.min() + 1e-12)
            ok &= int(qi[c] * periods.shape[0] + pi[c]) in ties
    out.append(("on-grid period injections are recovered", ok, ""))
    # P-Pdot: short periods, Pdot grid where a step dephases far beyond a bin
    ok = True
    for seed in range(4):
        periods = synth.log_periods(200.0, 260.0, 61)
        pdots = np.linspace(-1e-10, 0.0, 21)
        batch, pi, qi = synth.make_onegrid_injection(300 + seed, 2, 400, periods, pdots)
        grid = orc.ce_grid(batch.times, batch.mags, batch.offsets, batch.periods, batch.pdots,
                           15, 10)
        for c in range(batch.n_curves):
            g = grid[c].ravel()
            ties = np.flatnonzero(g <= g.min() + 1e-12)
            ok &= int(qi[c] * periods.shape[0] + pi[c]) in ties
    out.append(("on-grid (P, Pdot) injections are recovered", ok, ""))
    return out


def pin_overlapping_bins(orc):
    """50 %-overlapping phase bins (Sec. 2.3; the reading: bins of width 2/n_phase
    starting at j/n_phase).  Closed form: with two phase bins every point lies in
    both, so H is the Shannon entropy of the magnitude histogram.  Identity: the
    overlapping counts are the plain counts plus the plain counts of the next
    fine bin.  Bounds: 0 <= H <= ln n_mag."""
    rng = np.random.default_rng(41)
    out = []
    worst = 0.0
    for _ in range(40):
        n = int(rng.integers(5, 300))
        t = np.sort(rng.uniform(0, 1e8, n))
        m = rng.normal(15, 0.3, n)
        h, _, _ = orc.cell(t, m, 0.0, rng.uniform(200, 5000), -rng.uniform(0, 1e-10), 2, 10,
                           overlap=True)
        bins = orc.mag_bins(m, 10)
        worst = max(worst, abs(h - shannon(np.bincount(bins, minlength=10).astype(float))))
    out.append(("overlap, 2 phase bins: Shannon entropy of the magnitudes", worst < 1e-12,
                f"worst {worst:.3g}"))
    ok = True
    bounds = True
    for _ in range(60):
        n = int(rng.integers(2, 300))
        n_phase = int(rng.integers(2, 60))
        t = np.sort(rng.uniform(0, 1e8, n))
        m = rng.normal(15, 0.3, n)
        per, pd = rng.uniform(200, 5000), -rng.uniform(0, 1e-10)
        h1, c1, _ = orc.cell(t, m, 0.0, per, pd, n_phase, 10)
        h2, c2, _ = orc.cell(t, m, 0.0, per, pd, n_phase, 10, overlap=True)
        ok &= np.array_equal(c2, c1 + np.roll(c1, -1, axis=1))
        bounds &= -1e-15 <= h2 <= np.log(10) + 1e-12
        ok &= abs(h2 - chain_rule_entropy(c2)) < 1e-12
    out.append(("overlap counts are plain counts plus the next fine bin's", ok, ""))
    out.append(("overlap: 0 <= H <= ln n_mag", bounds, ""))
    return out


def pin_significance(orc):
    """Eq. 5 significance and Sec. 3.2's findings: a 7-minute chirping binary
    observed weekly for ten years (Sec. 2.2, Fig. 2) reaches the detection
    threshold rho = 10 only when the search has a Pdot axis, with a large gain in
    rho; a pure-noise light curve stays well below the threshold."""
    import oracle as oracle_mod
    rng = np.random.default_rng(43)
    base = 10 * 365.25 * 86400.0
    t = np.cumsum(rng.normal(7 * 86400.0, 86400.0, 521))
    t = np.sort(t - t[0])
    p0 = 420.0
    pdots = -np.geomspace(1e-12, 1e-10, 32)  # the Pdot axis of Sec. 3
    pd_true = pdots[20]
    df = 1.0 / (3.0 * base)                   # Sec. 3 frequency step, 1/(3B)
    periods = 1.0 / (1.0 / p0 + df * np.arange(-100, 101))
    cyc = synth.lightcurves.chirp_cycles(t, p0, pd_true)
    m = 16.0 + synth.lightcurves.eclipse_signal(cyc, 0.6, 0.05, 0.3) + rng.normal(0, 0.02, t.size)
    offs = np.array([0, t.size], dtype=np.int64)
    g_pd = orc.ce_grid(t, m, offs, periods, pdots, 15, 10)
    g_0 = orc.ce_grid(t, m, offs, periods, np.array([0.0]), 15, 10)
    _, _, r_pd = oracle_mod.oracle_significance(g_pd)
    _, _, r_0 = oracle_mod.oracle_significance(g_0)
    out = [("Eq. 5: the chirping 7-min binary is detected (rho > 10) with a Pdot axis",
            r_pd[0] > 10.0, f"rho {r_pd[0]:.2f}"),
           ("Sec. 3.2: rho gains more than 10 from the Pdot axis", r_pd[0] - r_0[0] > 10.0,
            f"rho {r_pd[0]:.2f} vs {r_0[0]:.2f}")]
    noise = 16.0 + rng.normal(0, 0.02, t.size)
    g_n = orc.ce_grid(t, noise, offs, periods, np.array([0.0]), 15, 10)
    mu, sd, r_n = oracle_mod.oracle_significance(g_n)
    flat = g_n.ravel()
    out.append(("Eq. 5 definition: rho = (mean - min) / population std",
                abs(r_n[0] - (flat.mean() - flat.min()) / flat.std()) < 1e-12, ""))
    out.append(("pure noise stays below the rho = 10 threshold", r_n[0] < 10.0,
                f"rho {r_n[0]:.2f}"))
    return out


def pin_band_normalization(orc):
    """Multi-filter input (Sec. 2.3): every filter of a curve is normalised on its
    own (median subtracted, divided by the standard deviation).  Library routine:
    numpy's median and population standard deviation per filter.  Closed form: a
    second filter that repeats every observation through an exact calibration
    (2 m + 3, dyadic data, 64 points, so every step is exact) normalises to the
    same values, and a curve whose every point is seen twice has the one-filter
    curve's CE grid bit for bit."""
    rng = np.random.default_rng(47)
    out = []
    worst = 0.0
    for _ in range(40):
        n = int(rng.integers(1, 200))
        nb = int(rng.integers(1, 5))
        m = rng.normal(15, 0.5, n)
        b = rng.integers(0, nb, n).astype(np.uint8)
        z = orc.band_normalize(m, b, [0, n], nb)
        for k in range(nb):
            x = m[b == k]
            if x.size == 0:
                continue
            sd = x.std()
            ref = (x - np.median(x)) / sd if sd > 0 else np.zeros_like(x)
            worst = max(worst, float(np.max(np.abs(z[b == k] - ref))))
    out.append(("filters: numpy median and population std per filter", worst < 1e-12,
                f"worst {worst:.3g}"))
    const = orc.band_normalize(np.full(5, 14.5), np.zeros(5, np.uint8), [0, 5], 1)
    out.append(("filters: a filter without spread normalises to 0", np.all(const == 0.0), ""))
    n = 64
    t = np.sort(rng.uniform(0.0, 1e8, n))
    m0 = np.round(rng.normal(15.0, 0.3, n) * 1024.0) / 1024.0
    per = synth.log_periods(300.0, 3000.0, 300)
    pd = np.array([0.0, -1e-11])
    z1 = orc.band_normalize(m0, np.zeros(n, np.uint8), [0, n], 1)
    g1 = orc.ce_grid(t, z1, np.array([0, n]), per, pd, 15, 10)
    b2 = np.r_[np.zeros(n), np.ones(n)].astype(np.uint8)
    z2 = orc.band_normalize(np.r_[m0, 2.0 * m0 + 3.0], b2, [0, 2 * n], 2)
    g2 = orc.ce_grid(np.r_[t, t], z2, np.array([0, 2 * n]), per, pd, 15, 10)
    out.append(("filters: an affine copy in a second filter normalises identically",
                np.array_equal(z2[:n], z2[n:]) and np.array_equal(z2[:n], z1), ""))
    out.append(("filters: every point seen twice leaves the CE grid unchanged",
                np.array_equal(g1, g2), f"max diff {np.abs(g1 - g2).max():.3g}"))
    return out


def pin_selection(orc):
    """Selection and Eq. 5 on grids with known answers.  Top-k: brute force over
    (H, flat index) pairs with Python's tuple order on grids full of ties, so
    equal H go to the smaller flat index q * n_periods + p.  Significance: a grid
    holding 0, 1, ..., n - 1 in any order has mean (n - 1)/2, population variance
    (n^2 - 1)/12 and minimum 0; a flat grid has rho = 0."""
    import oracle as oracle_mod
    rng = np.random.default_rng(53)
    ok = True
    for _ in range(30):
        n_c, n_q, n_p = (int(v) for v in rng.integers(1, 6, 3))
        k = int(rng.integers(1, n_q * n_p + 1))
        grid = rng.integers(0, 3, (n_c, n_q, n_p)).astype(np.float64)
        h, idx = oracle_mod.oracle_topk(grid, k)
        for c in range(n_c):
            pairs = sorted((grid[c, q, p], q * n_p + p) for q in range(n_q) for p in range(n_p))
            ok &= [i for _, i in pairs[:k]] == list(idx[c])
            ok &= [v for v, _ in pairs[:k]] == list(h[c])
    out = [("top-k: k smallest by (H, flat index), ties to the smaller index", bool(ok), "")]
    worst = 0.0
    for n in (2, 3, 10, 97, 1000):
        grid = rng.permutation(n).astype(np.float64).reshape(1, 1, n)
        mu, sd, rho = oracle_mod.oracle_significance(grid)
        want_sd = ((n * n - 1) / 12.0) ** 0.5
        worst = max(worst, abs(mu[0] - (n - 1) / 2.0), abs(sd[0] - want_sd) / want_sd,
                    abs(rho[0] - (n - 1) / 2.0 / want_sd))
    _, _, flat_rho = oracle_mod.oracle_significance(np.full((1, 2, 3), 0.7))
    out.append(("Eq. 5 on 0..n-1: mean (n-1)/2, population variance (n^2-1)/12",
                worst < 1e-12, f"worst {worst:.3g}"))
    out.append(("Eq. 5 on a flat grid: rho = 0", flat_rho[0] == 0.0, ""))
    return out


def pin_batch_paths(orc):
    """The batch paths against the single-cell path (itself pinned to exact
    arithmetic above): on a ragged batch with t0 != 0 and several Pdot values, the
    full grid (any thread count) and the sampled cells (with their counts) equal
    cell() at every (curve, q, p), with plain and overlapping bins, so curve
    offsets and the flat index q * n_periods + p are taken right."""
    rng = np.random.default_rng(59)
    lengths = [1, 2, 17, 64, 130]
    t = np.concatenate([np.sort(rng.uniform(0, 5e7, n)) for n in lengths])
    m = rng.normal(15, 0.3, t.size)
    offs = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    periods = np.exp(rng.uniform(np.log(300), np.log(3000), 23))
    pdots = np.array([0.0, -4e-11, 2e-11])
    t0 = 1.25e7
    n_p, n_q, n_c = periods.size, pdots.size, len(lengths)
    out = []
    for overlap in (False, True):
        grid = orc.ce_grid(t, m, offs, periods, pdots, 9, 7, t0=t0, n_threads=1,
                           overlap=overlap)
        grid4 = orc.ce_grid(t, m, offs, periods, pdots, 9, 7, t0=t0, n_threads=4,
                            overlap=overlap)
        cc = np.repeat(np.arange(n_c), n_p * n_q)
        ct = np.tile(np.arange(n_p * n_q), n_c)
        hc, _, counts = orc.ce_cells(t, m, offs, periods, pdots, 9, 7, cc, ct, t0=t0,
                                     with_counts=True, overlap=overlap)
        ok = np.array_equal(grid, grid4)
        ok &= np.array_equal(hc, grid.reshape(-1))
        for c in range(n_c):
            tc, mc = t[offs[c]:offs[c + 1]], m[offs[c]:offs[c + 1]]
            for q in range(n_q):
                for p_ in range(n_p):
                    h1, c1, _ = orc.cell(tc, mc, t0, periods[p_], pdots[q], 9, 7,
                                         overlap=overlap)
                    k = (c * n_q + q) * n_p + p_
                    ok &= h1 == grid[c, q, p_] and np.array_equal(c1, counts[k])
        out.append((f"batch grid and sampled cells equal the single-cell path"
                    f"{' (overlapping bins)' if overlap else ''}", bool(ok), ""))
    return out


ALL_PINS = (
    pin_fold_exact_rational, pin_fold_edges, pin_pdot_zero_plain_fold, pin_eq6_dephasing,
    pin_mag_bins, pin_entropy_chain_rule, pin_entropy_special_cases,
    pin_entropy_bounds_and_invariance, pin_brute_force_tiny, pin_paper_worked_example,
    pin_recovery, pin_overlapping_bins, pin_significance, pin_band_normalization,
    pin_selection, pin_batch_paths,
)


def run_all(orc):
    results = []
    for pin in ALL_PINS:
        results.extend(pin(orc))
    return results
