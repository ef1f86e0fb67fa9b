"""Comparison rules between the CUDA path and the FP64 oracle.

Aggregated costs: |Agg_gpu - Agg_oracle| / R <= 1e-5 with R the cost range
(2 for NCC, tau for TAD).

Integer disparities: identical, except at near ties -- pixels whose oracle
best and second-best aggregated costs differ by less than 4x the absolute
aggregated-cost tolerance.  There the GPU's choice must itself be within that
margin of the oracle's best (a valid winner); such pixels are counted.

Subpixel disparities: within 1e-3 px wherever the parabola of Eq. (10) is
well conditioned, i.e. where first-order propagation of the measured
aggregated-cost error through Eq. (10) stays below 1e-3 px.  Ill-conditioned
pixels (nearly flat parabolas) are counted and must still lie in the half-open
unit interval around the shared integer winner.
"""

from __future__ import annotations

import numpy as np

AGG_REL_TOL = 1e-5
SUBPIX_TOL = 1e-3


def agg_tolerance(cost_range):
    return AGG_REL_TOL * cost_range


def check_agg(agg_gpu, agg_ref, cost_range):
    err = np.abs(np.asarray(agg_gpu, np.float64) - np.asarray(agg_ref, np.float64))
    worst = float(err.max()) if err.size else 0.0
    assert worst <= agg_tolerance(cost_range), f"max |dAgg| = {worst:.3e} > {agg_tolerance(cost_range):.3e}"
    return worst


def near_tie_mask(agg_ref, margin):
    a = np.asarray(agg_ref, np.float64)
    if a.shape[-1] < 2:
        return np.zeros(a.shape[:-1], bool)
    part = np.partition(a, 1, axis=-1)
    return (part[..., 1] - part[..., 0]) < margin


def check_disparities(di_gpu, ds_gpu, agg_ref, di_ref, ds_ref, cost_range, agg_err=None, tol=None):
    """Returns a dict of counts; raises AssertionError on a violation.

    tol (optional): an absolute bound on |Agg_gpu - Agg_oracle| that replaces
    the FP32 tolerance (the 16-bit forms pass their rounding bound).  Then the
    near-tie margin is 2 tol, and every subpixel disparity whose parabola is
    defined under perturbations of tol must lie within the propagated bound
    of the oracle's (below) instead of within 1e-3 px."""
    a = np.asarray(agg_ref, np.float64)
    di_gpu = np.asarray(di_gpu).astype(np.int64)
    di_ref = np.asarray(di_ref).astype(np.int64)
    ds_gpu = np.asarray(ds_gpu, np.float64)
    ds_ref = np.asarray(ds_ref, np.float64)
    margin = 4.0 * agg_tolerance(cost_range) if tol is None else 2.0 * tol
    ties = near_tie_mask(a, margin)
    D = a.shape[-1]
    assert di_gpu.min() >= 0 and di_gpu.max() < D
    mismatch = di_gpu != di_ref
    bad = mismatch & ~ties
    assert not bad.any(), f"{int(bad.sum())} integer disparities differ away from near ties"
    # at near ties the GPU winner must be a valid (near-optimal) choice
    chosen = np.take_along_axis(a, di_gpu[..., None], -1)[..., 0]
    assert np.all(chosen - a.min(-1) <= margin + 1e-15)
    # subpixel: only where both sides chose the same winner
    same = ~mismatch
    b = di_ref
    interior = same & (b > 0) & (b < D - 1)
    bm = np.clip(b - 1, 0, D - 1)
    bp = np.clip(b + 1, 0, D - 1)
    Am = np.take_along_axis(a, bm[..., None], -1)[..., 0]
    A0 = np.take_along_axis(a, b[..., None], -1)[..., 0]
    Ap = np.take_along_axis(a, bp[..., None], -1)[..., 0]
    den = 2 * Am + 2 * Ap - 4 * A0
    err = np.abs(ds_gpu - ds_ref)
    off = ds_gpu[same] - di_gpu[same]
    assert np.all(off > -0.5 - 1e-6) and np.all(off <= 0.5 + 1e-6)
    if tol is None:
        eps = max(float(agg_err) if agg_err is not None else agg_tolerance(cost_range), 1e-7)
        with np.errstate(divide="ignore", invalid="ignore"):
            bound = 4 * eps * (np.abs(Ap - A0) + np.abs(Am - A0) + np.abs(Am - Ap)) / den ** 2
        well = same & (~interior | (bound < SUBPIX_TOL))
        assert np.all(err[well] <= SUBPIX_TOL), f"subpixel error {err[well].max():.3e} > {SUBPIX_TOL}"
        return dict(pixels=int(di_gpu.size), near_ties=int(ties.sum()), tie_mismatch=int((mismatch & ties).sum()),
                    ill_conditioned=int((same & ~well).sum()),
                    max_subpix_err=float(err[well].max()) if well.any() else 0.0)
    # Eq. (10) offset n / m with n = A- - A+, m = 2 A- + 2 A+ - 4 A0; each A
    # moved by at most tol moves n by 2 tol and m by 8 tol, so where m > 8 tol
    # |n'/m' - n/m| <= (2 tol |m| + 8 tol |n|) / (|m| (|m| - 8 tol))
    n = Am - Ap
    defined = interior & (den > 8 * tol)
    with np.errstate(divide="ignore", invalid="ignore"):
        pbound = (2 * tol * np.abs(den) + 8 * tol * np.abs(n)) / (np.abs(den) * (np.abs(den) - 8 * tol))
    chk = defined | (same & ~interior)
    limit = np.where(defined, pbound, 0.0) + 1e-5
    assert np.all(err[chk] <= limit[chk]), f"subpixel error beyond the propagated bound: {(err - limit)[chk].max():.3e}"
    return dict(pixels=int(di_gpu.size), near_ties=int(ties.sum()), tie_mismatch=int((mismatch & ties).sum()),
                undefined=int((same & interior & ~defined).sum()),
                max_subpix_err=float(err[chk].max()) if chk.any() else 0.0,
                median_subpix_bound=float(np.median(pbound[defined])) if defined.any() else 0.0)
