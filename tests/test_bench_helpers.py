"""Host-side helpers of bench.py on the CPU: the ncu launch-list summary that
the committed profile tables come from, and the ALU roofline arithmetic."""
import io
import os
import sys
from contextlib import redirect_stdout

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

HEADER = '"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size","Grid Size",' \
         '"Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"\n'


def _row(i, name, unit, value, metric="gpu__time_duration.sum"):
    return f'"{i}","1","python3","h","{name}","1","7","(256, 1, 1)","(1, 1, 1)","0","10.3","s","{metric}",' \
           f'"{unit}","{value}"\n'


def test_launch_summary_takes_the_launches_between_the_two_torch_kernels(tmp_path):
    """Only the launches after the first torch kernel (the L2-flush fill) and
    before the next one count; times are converted to microseconds, other
    metrics and ncu's own log lines are ignored, kernels are grouped by name
    and sorted by total time."""
    lines = ["==PROF== Connected to process\n", HEADER,
             _row(0, "void afd::stencil2_kernel<8, 2, 0>(afd::StencilArgs<float, float>)", "ns", "1,000"),
             _row(1, "void at::native::vectorized_elementwise_kernel<4, FillFunctor<float>>(int)", "ns", "500"),
             _row(2, "void afd::stencil2_kernel<8, 2, 0>(afd::StencilArgs<float, float>)", "usecond", "30"),
             _row(3, "void afd::k_update<float>(int, int)", "ns", "12,000"),
             _row(3, "void afd::k_update<float>(int, int)", "byte", "999", metric="dram__bytes_read.sum"),
             _row(4, "void afd::stencil2_kernel<8, 2, 0>(afd::StencilArgs<float, float>)", "usecond", "28"),
             _row(5, "void at::native::vectorized_elementwise_kernel<4, FillFunctor<float>>(int)", "ns", "500"),
             _row(6, "void afd::k_update<float>(int, int)", "ns", "90,000")]
    p = tmp_path / "launches.csv"
    p.write_text("".join(lines))
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.launch_summary(str(p))
    out = buf.getvalue().splitlines()
    assert out[0].startswith("launches in the timed step: 3, total device time 70.0 us")
    rows = [ln.split() for ln in out[2:]]
    assert rows[0][0].startswith("afd::stencil2_kernel<8,") and rows[0][-3:] == ["2", "58.0", "82.9%"]
    assert rows[1][0] == "afd::k_update<float>" and rows[1][-3:] == ["1", "12.0", "17.1%"]


def test_alu_roofline_arithmetic():
    r = bench.alu_roofline(1_000_000, 0.01)             # 147 MFLOP in 10 us
    assert r["flops_per_launch"] == 147_000_000
    assert abs(r["achieved"] - 14.7) < 1e-9
    peak = bench.fp32_peak_tflops(r["sm_count"], bench.sm_max_mhz())
    assert abs(r["peak"] - round(peak, 1)) < 1e-9
    assert abs(r["frac"] - 14.7 / peak) < 1e-4
    assert r["unit"] == "TFLOP/s" and r["bound"] == "alu"


def test_fp32_peak_from_unit_counts():
    # 152 SMs x 128 lanes x 2 flops x 2070 MHz
    assert abs(bench.fp32_peak_tflops(152, 2070.0) - 80.54) < 0.01
    assert abs(bench.fp32_peak_tflops(76, 2070.0) - 40.27) < 0.01
