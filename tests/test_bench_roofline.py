"""bench.py's roofline inputs from the committed ncu summaries: a recorded figure
(DRAM bytes per launch, instructions per update) counts only while the sources that
define its kernel are the ones it was captured from, and the register-resident FP64
kernel's ceiling is the busier of its two pipes."""
import os
import shutil

import bench


SRC = os.path.join(bench.ROOT, "paper_1811_08282_gb300", "csrc")


def _tree(tmp_path, traffic_lines):
    csrc = tmp_path / "paper_1811_08282_gb300" / "csrc"
    csrc.mkdir(parents=True)
    src = SRC
    for f in bench.KERNEL_SOURCES["k_heat_fold"]:
        shutil.copy(os.path.join(src, f), csrc / f)
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.txt").write_text("\n".join(traffic_lines) + "\n")
    return csrc


def test_recorded_figures_follow_the_kernel_sources(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    csrc = _tree(tmp_path, ["# comment", "k_heat_fold.source_sha=0000000000000000",
                            "k_heat_fold.heat_fp64.n2^24.bytes_per_launch=1000"])
    assert bench.recorded_traffic("k_heat_fold", "k_heat_fold.heat_fp64.n2^24") is None  # hash differs
    sha = bench.kernel_source_sha("k_heat_fold")
    (tmp_path / "profiles" / "traffic.txt").write_text(
        f"k_heat_fold.source_sha={sha}\nk_heat_fold.heat_fp64.n2^24.bytes_per_launch=1000\n"
        "k_heat_fold.heat_fp64.w128.alu_inst_per_update=51.5\n")
    assert bench.recorded_traffic("k_heat_fold", "k_heat_fold.heat_fp64.n2^24") == 1000.0
    assert bench.recorded("k_heat_fold", "k_heat_fold.heat_fp64.w128", "alu_inst_per_update") == 51.5
    assert bench.recorded("k_heat_fold", "k_heat_fold.heat_fp64.w256", "alu_inst_per_update") is None
    # any change to a defining source voids every recorded figure of the kernel
    with open(csrc / "fp64_soft.cuh", "a") as fh:
        fh.write("// edited\n")
    assert bench.kernel_source_sha("k_heat_fold") != sha
    assert bench.recorded_traffic("k_heat_fold", "k_heat_fold.heat_fp64.n2^24") is None
    assert bench.recorded("k_heat_fold", "k_heat_fold.heat_fp64.w128", "alu_inst_per_update") is None


def test_two_pipe_ceiling_takes_the_busier_pipe():
    # 3 FP64 instructions and nothing on the ALU pipe: the FP64 pipe alone, 5 flops per
    # update -> the FP64 peak (an FMA is 2 flops, the add 1: 5/6 of 2 flops per slot)
    fp64_only = min(bench.FP64_INST_PER_S / 3.0, bench.ALU_LANE_INST_PER_S / 1e-9)
    assert abs(fp64_only * 5 / 1e12 - bench.FP64_PEAK_TFLOPS * 5 / 6) < 1e-9
    # the committed counts of the mixed kernel: the ALU pipe binds, a little below the FP64 pipe
    f, a = 1.5562, 51.117
    assert bench.ALU_LANE_INST_PER_S / a < bench.FP64_INST_PER_S / f
    ceiling = min(bench.FP64_INST_PER_S / f, bench.ALU_LANE_INST_PER_S / a)
    assert 390e9 < ceiling < 398e9


def test_committed_counts_are_current_for_every_recorded_kernel():
    # every kernel with recorded ncu figures must still have the sources they were taken from,
    # or the bench line would drop its traffic and instruction counts (null)
    path = os.path.join(bench.ROOT, "profiles", "traffic.txt")
    shas = {}
    for line in open(path):
        line = line.strip()
        if line and not line.startswith("#") and ".source_sha=" in line:
            k, v = line.split(".source_sha=")
            shas[k] = v
    assert {"k_heat_fold", "k2d"} <= set(shas)
    for kernel, sha in shas.items():
        assert bench.kernel_source_sha(kernel) == sha, kernel


def test_2d_ceiling_is_the_busier_pipe_for_the_recorded_mix():
    fp64_rate, alu_rate = 528.8e9, 16.05e12
    ceil, f, a = bench.pipe_ceiling2d("k2d.phase_fp64.w64", fp64_rate, alu_rate)
    assert ceil == min(fp64_rate / f, alu_rate / a)
    assert 2.5 < f < 4.0 and 60 < a < 130  # about half the cells on each pipe
    assert 140e9 < ceil < 190e9
    step, f2, a2 = bench.pipe_ceiling2d("k2d.step_fp64", fp64_rate, alu_rate)
    assert step == min(fp64_rate / f2, alu_rate / a2)
    assert bench.pipe_ceiling2d("k2d.phase_fp64.w32", fp64_rate, alu_rate) == (None, None, None)
