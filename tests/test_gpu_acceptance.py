"""The pair search's acceptance test at the decision boundary.

A pair inside the cutoff reacts when its uniform u is below the probability p that the
pair's relative path touched the reaction sphere during the step (the absorbing-sphere
reading of Eq. kdiff1 and Eq. PDF0). The search decides most pairs on an FP32 estimate of
p with a worst-case error band and forms u and p in FP64 only inside the band, so its
decision must always be the FP64 decision. Here u is known in advance (its Philox block is
keyed by the pair and the step), the end separation d1 is solved so that p(d0, d1) = u,
and d1 is then stepped by single ulps across that crossing: every tiered decision of both
precisions must equal u < p in FP64, and the FP64 decisions must equal the reference's
wherever u and p differ by more than the last few bits. Runs through the C ABI."""
import numpy as np
import pytest

from harness import cuda_available
from oracle import sbs
from paper_2509_03313_gb300 import chem, workloads as W

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not cuda_available(), reason="needs a CUDA GPU")]

SEED, TRAIN = 0x1234_5678_9ABC, 3


def _context():
    import torch
    cfg, keep = chem.make_config(1000.0, W.D_NM2_S, W.WATER_REACTIONS, seed=SEED, train_id=TRAIN,
                                 precision=chem.CHEM_FP64, capacity_species=64,
                                 stream=torch.cuda.current_stream().cuda_stream)
    return chem.chem_init(cfg), keep


def _radii():
    R = np.array([sbs.reaction_radius(r.k_tab, W.D_NM2_S[r.a] + W.D_NM2_S[r.b]) for r in W.WATER_REACTIONS])
    DAB = np.array([W.D_NM2_S[r.a] + W.D_NM2_S[r.b] for r in W.WATER_REACTIONS])
    return R, DAB


def _solve_d1(d0, u, R, ddt):
    """d1 > R with touch_probability(d0, d1) = u (p falls from 1 to 0 as d1 grows)."""
    lo, hi = R, R + 60.0 * np.sqrt(ddt)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if mid == lo or mid == hi:
            break
        if sbs.touch_probability(d0, mid, R, ddt) > u:
            lo = mid
        else:
            hi = mid
    return lo


def _boundary_cases(rng, n_pairs, step, dt, float_inputs):
    R, DAB = _radii()
    key = sbs.philox_key(SEED, TRAIN)
    d0s, d1s, rx, los, his = [], [], [], [], []
    for _ in range(n_pairs):
        r = int(rng.integers(0, len(R)))
        lo = int(rng.integers(0, 1 << 28))
        hi = lo + 1 + int(rng.integers(0, 1 << 20))
        u = float(sbs.acceptance_uniform(np.array([lo]), np.array([hi]), step, key)[0])
        ddt = DAB[r] * dt
        if not (1e-300 < u < 1.0):
            continue
        # start separations from just outside R to several diffusion lengths
        d0 = R[r] + float(rng.choice([1e-3, 0.05, 0.3, 1.0, 2.5])) * np.sqrt(ddt) * float(rng.uniform(0.5, 1.5))
        d1 = _solve_d1(d0, u, R[r], ddt)
        if float_inputs:
            # FP32-local test: the inputs are FP32 squared separations
            c = np.float32(d1 * d1)
            steps = [c]
            for _ in range(6):
                steps.append(np.nextafter(steps[-1], np.float32(np.inf)))
            down = [c]
            for _ in range(6):
                down.append(np.nextafter(down[-1], np.float32(0)))
            d1sq = np.array(sorted(set(steps + down)), dtype=np.float64)
            d0sq = np.full(d1sq.shape, float(np.float32(d0 * d0)))
        else:
            d1v = [d1]
            for _ in range(8):
                d1v.append(np.nextafter(d1v[-1], np.inf))
            x = d1
            for _ in range(8):
                x = np.nextafter(x, 0.0)
                d1v.append(x)
            d1sq = np.array(d1v) ** 2
            d0sq = np.full(d1sq.shape, d0 * d0)
        d0s.append(d0sq)
        d1s.append(d1sq)
        rx.append(np.full(d1sq.shape, r))
        los.append(np.full(d1sq.shape, lo))
        his.append(np.full(d1sq.shape, hi))
    return (np.concatenate(d0s), np.concatenate(d1s), np.concatenate(rx).astype(np.int32),
            np.concatenate(los).astype(np.uint32), np.concatenate(his).astype(np.uint32))


def _wide_cases(rng, n, dt):
    # separations over the whole cutoff range, including inside R and far tails
    R, DAB = _radii()
    r = rng.integers(0, len(R), n)
    s = np.sqrt(DAB[r] * dt)
    d0 = R[r] * rng.uniform(0.5, 1.0, n) + rng.exponential(1.5, n) * s
    d1 = R[r] * rng.uniform(0.5, 1.0, n) + rng.exponential(1.5, n) * s
    lo = rng.integers(0, 1 << 28, n)
    hi = lo + 1 + rng.integers(0, 1 << 20, n)
    return d0 * d0, d1 * d1, r.astype(np.int32), lo.astype(np.uint32), hi.astype(np.uint32)


def _oracle_decisions(d0sq, d1sq, rxn, lo, hi, step, dt):
    R, DAB = _radii()
    key = sbs.philox_key(SEED, TRAIN)
    u = sbs.acceptance_uniform(lo.astype(np.uint64), hi.astype(np.uint64), step, key)
    p = sbs.touch_probability(np.sqrt(d0sq), np.sqrt(d1sq), R[rxn], DAB[rxn] * dt)
    return u, p


@pytest.mark.parametrize("precision", [chem.CHEM_FP64, chem.CHEM_FP32_LOCAL])
@pytest.mark.parametrize("dt", [1e-12, 1e-9, 3e-7])
def test_tiered_acceptance_equals_fp64_at_the_boundary(precision, dt):
    rng = np.random.default_rng(17 + int(precision))
    step = 41
    f32 = precision == chem.CHEM_FP32_LOCAL
    cases = [_boundary_cases(rng, 300, step, dt, f32), _wide_cases(rng, 200_000, dt)]
    ctx, keep = _context()
    try:
        for k, (d0sq, d1sq, rxn, lo, hi) in enumerate(cases):
            tiered, exact = chem.chem_check_acceptance(ctx, precision, step, dt, d0sq, d1sq, rxn, lo, hi)
            bad = np.nonzero(tiered != exact)[0]
            assert bad.size == 0, (f"case set {k}: {bad.size} tiered decisions differ from FP64, first "
                                   f"d0sq={d0sq[bad[0]]!r} d1sq={d1sq[bad[0]]!r} rxn={rxn[bad[0]]}")
            # the FP64 decision is the reference's wherever u and p are not within a few ulp
            if f32:
                d0sq = d0sq.astype(np.float32).astype(np.float64)
                d1sq = d1sq.astype(np.float32).astype(np.float64)
            u, p = _oracle_decisions(d0sq, d1sq, rxn, lo, hi, step, dt)
            clear = np.abs(u - p) > 1e-13 * np.maximum(p, 1e-300)
            assert np.array_equal(exact[clear], (u < p)[clear])
            if k == 0:
                # the boundary sets really straddle the crossing: both outcomes occur
                assert exact.any() and not exact.all()
                assert (~clear).sum() > 0 or f32
            else:
                assert 0 < exact.sum() < exact.size
    finally:
        chem.chem_destroy(ctx)


def test_acceptance_check_rejects_bad_input():
    ctx, keep = _context()
    try:
        with pytest.raises(chem.ChemError):
            chem.chem_check_acceptance(ctx, chem.CHEM_FP64, 0, 1e-9, [1.0], [1.0], [9], [0], [1])
    finally:
        chem.chem_destroy(ctx)
