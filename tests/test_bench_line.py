"""bench.py on the CPU: the JSON line assembled from fake GPU results, with every key the
output contract asks for, the roofline arithmetic of the dominant kernel and of the smoother
(all levels and the fine level alone), and that the line serialises; the reference arm's
line; the mixed-vs-FP64 error definitions and the oracle's sub-block sampling."""
import argparse
import json

import numpy as np
import pytest

import bench


def _res():
    prof = {
        "newton_assemble": dict(launches=20, ms=700.0, bytes=20 * 212.0 * 256**3),
        "mg_rbgs": dict(launches=6000, ms=60.0, bytes=3.0e11),
        "mg_rbgs_fine": dict(launches=2000, ms=180.0, bytes=7.0e11),
        "cg_spmv_dot": dict(launches=140, ms=37.0, bytes=1.1e11),
    }
    stats = [dict(newton_iters=4, linear_iters=35, kernel_launches=2970) for _ in range(4)]
    return dict(value=5.6e7, ms=1190.0, stats=stats, prof=prof, fp64={"value": 4.1e7, "ms_per_step": 409.0, "speedup_mixed_vs_fp64": 1.37,
                                                           "newton_iters": [4] * 4, "linear_iters": [30] * 4,
                                                           "mixed_vs_fp64_error": {"E_rel_2": 1e-11}},
                clocks={"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": []},
                e2e={"value": 5.1e7, "unit": "cell-steps/s", "h2d_bytes_per_step": 1, "d2h_bytes_per_step": 1},
                w=None, advect={"advect": dict(launches=10, ms=16.3, bytes=10 * 72.0 * 256**3), "courant_max": 0.05})


def test_bench_line_contract_and_rooflines():
    args = argparse.Namespace(size=256, steps=4, warmup=3, newton_tol=1e-6, lin_rtol=1e-3)
    line = bench.bench_line(args, _res(), 1, {"hbm_gbs": 6797.2})
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "gpu_launches", "clocks", "e2e"):
        assert key in line, key
    roof = line["roofline"]
    assert roof["kernel"] == "newton_assemble" and roof["bound"] == "alu"
    assert roof["achieved"] == pytest.approx(bench.ASSEMBLE_FP64_FLOPS_PER_CELL * 256**3 / 0.035 / 1e12)
    assert roof["frac"] == pytest.approx(roof["achieved"] / roof["peak"])
    assert roof["traffic"] == pytest.approx(bench.ASSEMBLE_DRAM_BYTES_PER_CELL * 256**3)
    mg = line["roofline_vcycle_smoother"]
    assert mg["achieved"] == pytest.approx(1.0e12 / 8000 / (0.24 / 8000) / 1e9)          # all levels
    assert mg["fine_level"]["achieved"] == pytest.approx(7.0e11 / 0.180 / 1e9)
    assert mg["fine_level"]["frac"] == pytest.approx(mg["fine_level"]["achieved"] / 6797.2)
    assert line["gpu_launches"] == 4 * 2970 + 4
    assert line["ms_per_step"] == pytest.approx(1190.0 / 4)
    # the FP64 arm and the per-kernel shares sit in the config block
    cfg = line["config"]
    assert cfg["fp64_path"]["speedup_mixed_vs_fp64"] == 1.37 and cfg["mixed_vs_fp64_error"]["E_rel_2"] == 1e-11
    assert cfg["kernel_shares"]["newton_assemble"][0] == pytest.approx(700.0 / 1190.0, abs=1e-4)
    assert cfg["vcycle_smoother"]["fine_level"]["achieved"] == pytest.approx(mg["fine_level"]["achieved"])
    json.loads(json.dumps(line))


def test_config_describes_the_workload_at_each_size():
    """The workload and L2 notes follow the grid: 2000 sources and fields above L2 at 256^3
    (no flush needed); fewer sources and an honest 'not flushed' below."""
    for n, nsrc, above in ((256, 2000, True), (128, 2000, True), (64, 31, False)):
        args = argparse.Namespace(size=n, steps=4, warmup=3, newton_tol=1e-6, lin_rtol=1e-3)
        cfg = bench.bench_line(args, _res(), 1, {"hbm_gbs": 6797.2})["config"]
        assert f"{n}^3, {nsrc} sources" in cfg["workload"]
        assert cfg["l2"].startswith("inputs larger than L2" if above else "inputs smaller than L2")
        assert bench.workload_sources(n) == nsrc


def test_helium_option_uses_the_helium_kernel_figures():
    args = argparse.Namespace(size=128, steps=2, warmup=3, newton_tol=1e-6, lin_rtol=1e-3, helium=True)
    line = bench.bench_line(args, _res(), 1, {"hbm_gbs": 6797.2})
    assert "hydrogen + helium" in line["config"]["workload"]
    roof = line["roofline"]
    assert roof["flops_per_cell"] == bench.ASSEMBLE_HE_FP64_FLOPS_PER_CELL
    assert roof["traffic"] == pytest.approx(bench.ASSEMBLE_HE_DRAM_BYTES_PER_CELL * 128**3)


def test_reference_arm_line(capsys):
    """bench.py --impl reference: the oracle on host cores prints one JSON line with the
    contract's keys, a cpu_baseline describing the run and a zero-copy e2e."""
    args = argparse.Namespace(size=32, steps=1, warmup=0, newton_tol=1e-6, gpus=1)
    bench.run_reference(args)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == "cell-steps/s"
    assert line["value"] > 0 and line["higher_is_better"] is True and line["steps"] == 1
    cpu = line["cpu_baseline"]
    assert cpu["kind"] == "oracle" and cpu["cores"] >= 1 and cpu["value"] == line["value"] and cpu["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": "cell-steps/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_state_errors_definitions():
    """E normwise (2 and max) relative, x_HI pointwise relative with a 1e-8 floor, T pointwise."""
    Eb, xb, Tb = np.array([1.0, 2.0, 2.0]), np.array([1e-10, 0.5, 1.0]), np.array([100.0, 1e4, 1e4])
    Ea, xa, Ta = Eb + np.array([0.0, 0.0, 0.3]), xb + np.array([1e-9, 0.0, -0.1]), Tb * np.array([1.0, 1.01, 1.0])
    e = bench.state_errors((Ea, xa, Ta), (Eb, xb, Tb))
    assert e["E_rel_2"] == pytest.approx(0.3 / 3.0)
    assert e["E_rel_inf"] == pytest.approx(0.3 / 2.0)
    assert e["xHI_rel_max"] == pytest.approx(0.1)          # 1e-9 / max(1e-10, 1e-8) = 0.1 as well
    assert e["T_rel_max"] == pytest.approx(0.01)


def test_oracle_sample_is_the_sub_block_with_its_sources():
    import workloads as W
    w = W.reionization_field(n=16, nsrc=12, box_mpc=14.4 * 16 / 256)
    m = 8
    corner = bench.densest_corner(w, m)
    shape = (16, 16, 16)
    zc, yc, xc = np.unravel_index(w["src_index"], shape)
    counts = {}
    for z0 in (0, 8):
        for y0 in (0, 8):
            for x0 in (0, 8):
                counts[(z0, y0, x0)] = int(np.sum((zc // 8 == z0 // 8) & (yc // 8 == y0 // 8) & (xc // 8 == x0 // 8)))
    assert counts[corner] == max(counts.values())
    sub = bench.oracle_sample(w, m, corner)
    z0, y0, x0 = corner
    np.testing.assert_array_equal(sub["rho_b"], w["rho_b"][z0:z0 + m, y0:y0 + m, x0:x0 + m])
    assert sub["nx"] == sub["ny"] == sub["nz"] == m and sub["periodic"] == (True, True, True)
    assert len(sub["src_index"]) == counts[corner]
    # each sub-block source is the same cell, with the same rate, as in the full field
    sz, sy, sx = np.unravel_index(sub["src_index"], (m, m, m))
    full = np.ravel_multi_index((sz + z0, sy + y0, sx + x0), shape)
    for f, nd in zip(full, sub["src_ndot"]):
        k = int(np.flatnonzero(np.asarray(w["src_index"]) == f)[0])
        assert nd == w["src_ndot"][k]
