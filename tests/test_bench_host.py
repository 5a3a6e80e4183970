"""Host-side helpers of the benchmark (no GPU): time to target from the
bottom-right record of each event, its summary, and kernel naming."""
import numpy as np

import bench


def test_residual_tts_first_event_at_each_target():
    N, scale, E, interval = 10, 2.0, -1000, 50
    unit = N * scale  # one unit of residual energy per spin
    # run 0: feasible from event 2 on, residual 0.3, 0.15, 0.08, then at the planted energy
    # run 1: below every target but never feasible
    # run 2: feasible and at rho 0.2 exactly at event 4 (targets are inclusive), then nothing better
    f = np.array([[E + 0.05 * unit, E + 0.3 * unit, E + 0.15 * unit, E + 0.08 * unit, E, E],
                  [E - unit] * 6,
                  [E + unit, E + unit, E + unit, E + 0.2 * unit, E + 0.2 * unit, E + 0.2 * unit]])
    g = np.array([[1, 0, 0, 0, 0, 0], [2] * 6, [0] * 6])
    out = bench.residual_tts(f, g, 6, E, N, scale, interval)
    assert list(out["rho<=0.2"]) == [3 * interval, -1, 4 * interval]
    assert list(out["rho<=0.1"]) == [4 * interval, -1, -1]
    assert list(out["rho<=0.05"]) == [5 * interval, -1, -1]
    assert list(out["planted"]) == [5 * interval, -1, -1]
    # only the events run count
    out = bench.residual_tts(f, g, 4, E, N, scale, interval)
    assert list(out["planted"]) == [-1, -1, -1] and list(out["rho<=0.1"]) == [4 * interval, -1, -1]


def test_tts_summary_medians_and_censoring():
    per = {"rho<=0.2": np.array([100, 300, -1, 200]), "planted": np.array([-1, -1, -1, -1])}
    s = bench.tts_summary(per, 0.01)
    assert s["rho<=0.2"] == {"reached": 3, "runs": 4, "median_sweeps": 200.0, "median_seconds": 2.0}
    assert s["planted"]["reached"] == 0 and s["planted"]["median_sweeps"] is None
    assert s["planted"]["median_seconds"] is None


def test_sweep_kernel_names():
    assert bench.sweep_kernel_name({"kernel": "smem", "walkers_per_thread": 4}) == "k_sweep_smem"
    assert bench.sweep_kernel_name({"kernel": "bits", "walkers_per_thread": 8}) == "k_sweep_bits8"
    assert bench.sweep_kernel_name({"kernel": "bits", "walkers_per_thread": 4}) == "k_sweep_bits"
    assert bench.sweep_kernel_name({"kernel": "penalty_bits", "walkers_per_thread": 8}) == "k_sweep_penalty_bits8"
    assert bench.sweep_kernel_name({"kernel": "generic_smem", "walkers_per_thread": 4}) == "k_sweep_generic_smem"
