"""bench.py's compact end-of-line summary on CPU: built from a complete result
line, and from one whose extra parts failed, without raising."""
import json

import bench


def _line():
    return {
        "roofline": {"bound": "hbm", "frac": 0.14, "binding": "factor-row gathers served from L2",
                     "gather_bound": {"ms_per_mode": [0.84, 0.84, 0.89], "frac": 0.9,
                                      "rows_per_sm_clk_kernel": [0.3, 0.3, 0.3],
                                      "rows_per_sm_clk_bound": [0.33, 0.33, 0.33]}},
        "spttm": {"ms": 1.12, "GBps": 3650.0, "nfib": 51268194,
                  "idx16": {"ms": 1.07, "GBps": 3638.0, "speedup": 1.046}},
        "mttkrp_bf16": {"ms_per_step": 1.86, "GBps": 1496.0, "frac_of_gather_bound": 0.78},
        "cp_als": {"fp32": {"s_per_iter": 0.0056, "fit": 0.9862, "fit_diff_vs_oracle": 1.5e-7,
                            "factor_rel_vs_oracle": [0.004, 0.004, 0.025]},
                   "mixed": {"s_per_iter": 0.0039, "fit": 0.9862, "speedup_vs_fp32": 1.43},
                   "oracle_fp64": {"fit": 0.986205}},
        "sparse_fit": {"ms_per_step": 1.55, "loss_first": 1.98e7, "loss_last": 7.5e6, "noise_floor": 1000.0},
        "spttmc": {"ranks": [{"R": 16, "modes": [{"TFLOPs": 16.2}]}, {"R": 8, "modes": [{"TFLOPs": 9.0}]}]},
        "tucker": {"ms_per_iter": 9.3},
    }


def test_summary_of_a_complete_line():
    out = bench.summarize(_line())
    json.dumps(out)
    assert out["binding_roof"].startswith("factor-row gathers")
    assert out["spmttkrp_fp32_R32_gather_bound"]["frac"] == 0.9
    assert out["spmttkrp_bf16_R32"]["GBps"] == 1496.0
    assert out["cp_als_R64_20"]["mixed_speedup_vs_fp32"] == 1.43
    assert out["cp_als_R64_20"]["oracle_fit"] == 0.986205
    assert out["spttmc_mode0_TFLOPs"] == {"16": 16.2, "8": 9.0}
    assert out["tucker_R8_ms_per_iter"] == 9.3


def test_summary_of_failed_extras():
    line = _line()
    for k in ("spttm", "mttkrp_bf16", "cp_als", "sparse_fit", "spttmc", "tucker"):
        line[k] = {"error": "RuntimeError: failed"}
    out = bench.summarize(line)
    json.dumps(out)
    assert out["spttm_4way_mode3"]["GBps"] is None
    assert out["spttmc_mode0_TFLOPs"] == {}
