"""The CPU oracle's time-to-tol model in bench.py (OracleCost.predict) and its trajectories: host logic only.

The model sums the oracle's per-component times along a solve's iteration trajectory (kind and active columns per
iteration); these tests pin its bookkeeping, not the timings.
"""
import bench
import workloads as wl

UNIT = {k: 1.0 for k in bench.ORACLE_COMPONENTS}


def test_trajectory_summary_round_trip():
    kt = 40
    traj = [(0, 1, kt)] + [(it, 1 if it % 5 == 0 else 0, kt if it < 12 else 17) for it in range(1, 23)]
    back = bench.trajectory_expand(bench.trajectory_summary(traj), kt)
    assert back == traj


def test_predict_hand_sum():
    # kt = 10 columns; iteration 1 plain at full width, iteration 2 a Rayleigh-Ritz step with 5 active columns
    t = dict(UNIT, orth=2.0, rr=3.0)
    traj = [(0, 1, 10), (1, 0, 10), (2, 1, 5)]
    start = 2.0 + 3.0                                   # CholeskyQR2 of X0 and the initial Rayleigh-Ritz step
    it1 = (1 + 1) * 1.0 + 1 * 1.0 * 1 + 0.0 + (2.0 + 1) * 1.0 + 1 * 1.0     # precond+blocks, project once, copy 0,
    #                                                                           orth+resid (a^2), H (a)
    it2 = (1 + 1) * 0.5 + 1 * 0.5 * 2 + 1 * 0.5 + 3.0   # precond+blocks, project twice, copy of 5 locked, rr
    assert abs(bench.OracleCost.predict(t, traj, 10) - (start + it1 + it2)) < 1e-12


def test_predict_counts_a_repeated_final_step_once():
    # the solve history lists the final step twice; the model must price it once
    traj = [(0, 1, 8), (1, 0, 8), (2, 1, 8)]
    assert bench.OracleCost.predict(UNIT, traj + [(2, 1, 8)], 8) == bench.OracleCost.predict(UNIT, traj, 8)


def test_stored_48_trajectory_matches_the_workload():
    w = wl.GRID48_K1024
    kt = w.k + w.nbuf
    traj = bench.trajectory_expand(bench.TRAJECTORY_GRID48, kt)
    its = sorted({it for it, _, _ in traj})
    assert its == list(range(0, its[-1] + 1))           # every iteration from the start to the last
    assert traj[0] == (0, 1, kt) and traj[1][2] == kt    # full width at the start
    rr = sorted({it for it, kind, _ in traj if kind == 1 and it > 0})
    assert all(it % w.rr_period == 0 for it in rr[:-1])  # periodic Rayleigh-Ritz, plus the final step
    ka = [a for _, _, a in traj]
    assert all(x >= y for x, y in zip(ka, ka[1:]))       # locking only shrinks the active block
    assert min(ka) >= w.nbuf                              # buffer vectors never lock
