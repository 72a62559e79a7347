"""The bench's CPU legs on a tiny scene, without a GPU: the oracle baseline
estimators and their comparison with a GPU image (here the oracle's own
image, and the same image with one pixel moved)."""
import numpy as np

import oracle
import wsr_scenes as ws


def _tiny():
    sc = ws.random_scene(300, 5, sh_degree=1, vd_opacity=True, clusters=3, box=1.0, log_scale_mu=-3.0)
    cam = ws.look_at((0.1, 0.2, -3.0), width=40, height=30).rounded()
    w = ws.WeightParams(ws.EXP, 0.1, 0.8, 0.9, (0.1, 0.2, 0.3)).rounded()
    return sc, cam, w


def test_cpu_band_rate_compares_the_band_with_the_gpu_image():
    import bench
    sc, cam, w = _tiny()
    ref = oracle.render(sc, cam, w)["rgb"].astype(np.float32)
    res = bench.cpu_band_rate(sc, cam, w, 0.5, True, "a tiny scene", gpu_rgb=ref)
    assert res["kind"] == "oracle" and res["value"] > 0 and res["cores"] >= 1
    v = res["vs_oracle"]
    assert v["pixels_checked"] == cam.width * cam.height     # the taller band is the whole 30-row view
    assert v["max_abs_err"] < 1e-6                            # float32 rounding of the oracle's own image
    assert v["max_abs_err_beyond_tie_bound"] < 1e-6
    moved = ref.copy()
    moved[15, 20, 1] += 0.25
    v2 = bench.cpu_band_rate(sc, cam, w, 0.5, False, "a tiny scene", gpu_rgb=moved)["vs_oracle"]
    assert abs(v2["max_abs_err"] - 0.25) < 1e-6
    # one channel of one pixel off by 0.25: mse = 0.25^2 / (3 * 1200)
    assert abs(v2["psnr_db"] - 10 * np.log10(3 * 1200 / 0.0625)) <= 0.005     # reported to 0.01 dB
    assert "vs_oracle" not in bench.cpu_band_rate(sc, cam, w, 0.5, False, "a tiny scene")


def test_cpu_oracle_leg_reports_the_whole_view_and_its_error():
    import bench
    sc, cam, w = _tiny()
    target = ws.target_image(3, cam.height, cam.width)
    ref = oracle.render(sc, cam, w)["rgb"].astype(np.float32)
    base, err = bench.cpu_oracle_leg(sc, cam, w, target, ref, 0.5)
    assert base["kind"] == "oracle" and base["unit"] == "Mpix/s" and base["value"] > 0
    assert err["max_abs_err"] < 1e-6 and err["max_abs_err_beyond_tie_bound"] < 1e-6
    assert err["pixels_checked"] <= cam.width * cam.height


def _fake_nvidia_smi(tmp_path, lines):
    script = tmp_path / "nvidia-smi"
    body = "".join(f"printf '%s\\n' '{ln}'\n" for ln in lines)
    script.write_text("#!/bin/sh\n" + body + "exec sleep 30\n")
    script.chmod(0o755)


def test_clock_sampler_reads_clocks_and_throttle_reasons(tmp_path, monkeypatch):
    """The clocks record of the bench line from nvidia-smi's CSV samples: the
    median SM clock under load (idle samples below half the peak dropped),
    the maximum clock, and every throttle reason seen active."""
    import os

    import bench
    _fake_nvidia_smi(tmp_path, [
        "0, 345, 2070, 150.1, 0x0000000000000001, Not Active, Not Active, Not Active, Not Active",
        "0, 2070, 2070, 1010.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1390.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1200.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "malformed line"])
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ["PATH"])
    c = bench.ClockSampler(0)
    c.start()
    rec = c.stop()
    assert rec["sm_mhz"] == 2070.0 and rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == ["sw_power_cap"] and rec["samples"] == 4


def test_clock_sampler_reports_slowdowns_and_a_missing_tool(tmp_path, monkeypatch):
    import os

    import bench
    _fake_nvidia_smi(tmp_path, [
        "0, 1500, 2070, 1300.0, 0x0000000000000008, Active, Not Active, Not Active, Not Active",
        "0, 1450, 2070, 1300.0, 0x0000000000000008, Active, Active, Not Active, Not Active"])
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ["PATH"])
    c = bench.ClockSampler(0)
    c.start()
    rec = c.stop()
    assert rec["sm_mhz"] == 1475.0 and rec["reasons"] == ["hw_slowdown", "hw_thermal_slowdown"]
    empty = tmp_path / "empty"
    empty.mkdir()
    monkeypatch.setenv("PATH", str(empty))
    c = bench.ClockSampler(0)
    c.start()
    assert c.stop()["reasons"] == ["unavailable"]


def test_profile_traffic_is_dropped_when_the_kernel_source_changed(tmp_path, monkeypatch):
    """roofline.traffic comes from a committed ncu summary only while the
    render source it was captured from is unchanged (its sha256 recorded in
    the summary); after any change it is reported as null."""
    import hashlib

    import bench
    (tmp_path / "profiles").mkdir()
    src = tmp_path / "paper_2410_18931_gb300" / "csrc"
    src.mkdir(parents=True)
    (src / "render.cu").write_text("// kernel source\n")
    sha = hashlib.sha256((src / "render.cu").read_bytes()).hexdigest()
    (tmp_path / "profiles" / "k_render_bwd.md").write_text(
        f"# summary\n\ntraffic_bytes_per_launch: 264801792\nsource_sha256: {sha}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profile_traffic("k_render_bwd") == 264801792.0
    assert bench.profile_traffic("k_render_fwd") is None              # no summary
    (src / "render.cu").write_text("// kernel source, edited\n")
    assert bench.profile_traffic("k_render_bwd") is None


def test_launch_counts_claimed_per_step_match_the_profiled_launch_lists():
    """The bench's gpu_launches claim is kernels per step x steps; the kernels
    per step of each measured step (plain, deterministic, training; the
    persistent schedule) equal the launches of one step in its committed ncu
    launch list."""
    import os
    import re

    import __graft_entry__
    import bench
    __graft_entry__._build_module().build()       # the package loads its library on import
    from paper_2410_18931_gb300.train import TrainStep

    def profiled(name):
        text = open(os.path.join(bench.ROOT, "profiles", name)).read()
        return len(re.findall(r"^\| `k_\w+", text, flags=re.M))

    from paper_2410_18931_gb300 import _abi as A

    class _R:                                      # the count only: no device state
        # 1080p holds 16200 16x8 tiles or 8160 16x16 ones: one scan kernel (with the tile order)
        bin_kernels = 3
    assert 1920 // 16 * 1080 // 8 <= A.WSR_SCAN_ONE_BLOCK_TILES
    plain = bench.KERNELS_PER_STEP + _R.bin_kernels
    assert profiled("launches_1M_1080p.md") == plain
    assert profiled("launches_det_1M_1080p.md") == plain + 1 + 3          # the list sort; see run_deterministic
    step = TrainStep.__new__(TrainStep)
    step.r, step.persistent, step.deterministic = _R(), True, False
    assert profiled("launches_train_1M_1080p.md") == step.kernels_per_step
