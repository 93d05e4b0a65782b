"""Host logic of the pulse-train alternation (Sec. 2.1) and of the post-irradiation
analysis (Sec. 3.3), on the CPU: the call sequencing against a recording stand-in for the
library, and the analysis against closed forms and numpy's least squares."""
import numpy as np
import pytest

from paper_2509_03313_gb300 import hybrid, workloads as W


class _FakeChem:
    """Records the batched calls; each train's clock jumps to its end time."""

    def __init__(self, B):
        self.t = np.zeros(B)
        self.calls = []
        self.steps = np.zeros(B, np.int64)

    def chem_batch_run_until(self, ctx, ends):
        ends = np.asarray(ends, float)
        self.calls.append(("sbs", ends.copy()))
        adv = ends > self.t
        self.steps[adv] += 10
        self.t = np.where(adv, ends, self.t)

    def chem_batch_run_homogeneous(self, ctx, ends):
        ends = np.asarray(ends, float)
        self.calls.append(("ode", ends.copy()))
        self.t = np.where(ends > self.t, ends, self.t)

    def chem_batch_homogeneous_report(self, ctx, b):
        return np.full(16, 0.5), np.zeros(16, np.int64), 3

    def chem_batch_tally(self, ctx, b, n_types, n_rxn):
        c = np.zeros(8, np.int64)
        c[:3] = int(1e6 * self.t[b]) % 97
        return {"counts": c, "events": np.zeros(16, np.int64), "t": float(self.t[b]),
                "species_steps": int(self.steps[b])}


def test_plans_run_in_lockstep_and_trains_past_their_plan_idle(monkeypatch):
    fake = _FakeChem(3)
    monkeypatch.setattr(hybrid, "chem", fake)
    plans = [W.hybrid_stages(3, 1e-4, 1e-6, tail_s=10.0),
             W.hybrid_stages(2, 1e-3, 1e-6, tail_s=1.0),
             [("sbs", 5e-6)]]
    run = hybrid.run_plans(None, plans)
    # plans whose kinds differ at an index: both kinds run, each train in its own
    fake2 = _FakeChem(2)
    monkeypatch.setattr(hybrid, "chem", fake2)
    hybrid.run_plans(None, [[("sbs", 1.0), ("ode", 2.0)], [("ode", 1.5), ("sbs", 3.0)]])
    assert [(k, e.tolist()) for k, e in fake2.calls] == [
        ("sbs", [1.0, 0.0]), ("ode", [0.0, 1.5]), ("sbs", [0.0, 3.0]), ("ode", [2.0, 0.0])]
    monkeypatch.setattr(hybrid, "chem", fake)
    # one batched call per plan index (the plans alternate in step), none per train
    assert [k for k, _ in fake.calls] == ["sbs", "ode"] * 3
    # a train whose plan ended, or whose call is of the other kind, gets end time 0
    ends_sbs = [e for k, e in fake.calls if k == "sbs"]
    assert ends_sbs[0].tolist() == [1e-6, 1e-6, 5e-6]
    assert ends_sbs[-1][2] == 0.0
    np.testing.assert_array_equal(run["t"][-1], [plans[0][-1][1], plans[1][-1][1], 5e-6])
    assert run["kinds"][1] == ["ode", "ode", None]
    assert run["species_steps"] == int(fake.steps.sum())


def test_stoichiometry_of_the_water_table():
    nu = hybrid.stoichiometry(7, W.WATER_REACTIONS)
    # every reaction conserves charge; H and O balance with the water change
    water = np.array([rx.water_delta for rx in W.WATER_REACTIONS])
    assert np.all(W.CHARGE @ nu == 0)
    assert np.all(W.N_H @ nu + 2 * water == 0)
    assert np.all(W.N_O @ nu + water == 0)
    assert nu[:, 0].tolist() == [-2, 0, 0, 0, 2, 1, 0]  # R1: e + e -> H2 + 2 OH-


def test_hybrid_stages_cover_beam_on_and_off():
    plan = W.hybrid_stages(3, 2e-3, 1e-6, tail_s=10.0)
    assert plan == [("sbs", 1e-6), ("ode", 2e-3), ("sbs", 2e-3 + 1e-6), ("ode", 4e-3),
                    ("sbs", 4e-3 + 1e-6), ("ode", 4e-3 + 1e-6 + 10.0)]


def test_dose_slope_yield_is_the_least_squares_slope():
    rng = np.random.default_rng(0)
    dose = np.array([1.0, 5.0, 10.0, 15.0, 20.0])
    c = 2.7e-8 * dose + 1e-9 + rng.normal(0, 1e-10, size=5)
    slope, g = hybrid.dose_slope_yield(dose, c)
    assert slope == pytest.approx(np.polyfit(dose, c, 1)[0], rel=1e-12)
    # 1 molecule / 100 eV is 1.0364e-7 mol/J
    assert g == pytest.approx(slope / 1.0364e-7, rel=1e-4)
    s2, g2 = hybrid.dose_slope_yield([0.0, 1.0], [0.0, 1.0364e-7])
    assert g2 == pytest.approx(1.0, rel=1e-4)


def test_concentration_of_molecules_in_the_box():
    # 1 mol/L in a (1 um)^3 box (1e-15 L) holds N_A * 1e-15 molecules
    assert hybrid.concentration(6.02214076e8, 1000.0) == pytest.approx(1.0, rel=1e-12)


def test_buildup_fraction_and_threshold():
    kinds = [["sbs"] * 2, ["ode"] * 2, ["sbs"] * 2, ["ode"] * 2, ["sbs"] * 2, ["ode"] * 2]
    counts = np.zeros((6, 2, 7), np.int64)
    counts[2, :, 1] = [1000, 1000]   # end of the second pulse's beam-on stage
    counts[3, :, 1] = [3, 400]       # when the third pulse starts
    f = hybrid.buildup_fraction({"kinds": kinds, "counts": counts})
    np.testing.assert_allclose(f, [0.003, 0.4])
    # the real numbers left by the rate equations: counts before + nu @ extents
    extents = np.zeros((6, 2, 9))
    extents[3, 0, 5] = 499.9  # R6: OH + OH -> H2O2, 999.8 OH consumed of 1000
    nu = hybrid.stoichiometry(7, W.WATER_REACTIONS)
    f = hybrid.buildup_fraction({"kinds": kinds, "counts": counts, "extents": extents}, nu=nu)
    np.testing.assert_allclose(f, [0.0002, 1.0])
    assert hybrid.threshold_dose_rate([1.0, 1e4], f) == 1e4
    assert hybrid.threshold_dose_rate([1.0, 1e4], [0.0, 0.001]) is None
