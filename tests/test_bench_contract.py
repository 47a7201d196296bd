"""The bench's roofline arithmetic and kernel naming, on the CPU: every kernel the bench names
for a phase exists in the CUDA sources, the projection named is the one the solve dispatches
for 4 padded labels, and the reported fractions are the algorithmic work over the measured
time over the peak."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1607_04174_gb300", "csrc")


def _kernels():
    names = set()
    for f in os.listdir(CSRC):
        if f.endswith(".cu"):
            text = open(os.path.join(CSRC, f)).read()
            names |= set(re.findall(r"\b(k_[a-z0-9_]+)\s*\(", text))
    return names


def test_phase_kernels_exist():
    import bench
    defined = _kernels()
    for phase, spec in bench.PHASE_KERNELS.items():
        for part in spec.split("+"):
            name = part.split()[0]
            assert name in defined, (phase, name)
    for name in bench.NCU_DRAM_BYTES:
        assert name in defined, name


def test_projection_named_is_the_dispatched_one():
    """With at most 8 padded labels the 16-bit projection runs k_project_tma."""
    import bench
    text = open(os.path.join(CSRC, "solve.cu")).read()
    i = text.index("if (!back) {")
    branch = text[i:i + 900]
    assert "if constexpr (LP <= 8)" in branch
    assert branch.index("k_project_tma") < branch.index("k_project_cw")
    assert bench.PHASE_KERNELS["project"].startswith("k_project_tma")


def test_roofline_arithmetic():
    import bench
    N, m, lp, S, L, steps = 512 * 512, 84, 4, 800, 4, 3
    phases = {"seeds": 0.009, "gather": 0.027, "adapt": 0.049, "project": 0.024,
              "small": 0.019, "back": 0.016, "refine": 0.016}
    top, table = bench.rooflines(phases, N, m, lp, S, L, steps, hbm=6774.0, sm_mhz=2070.0)
    # the dominant phase is the longest one, with the captured traffic of its kernel (null when
    # the kernel has changed since its last capture)
    assert top["phase"] == "adapt" and top["kernel"] == "k_adapt_lu"
    assert top["traffic"] == bench.NCU_DRAM_BYTES.get("k_adapt_lu")
    alu = 152 * 128 * 2 * 2070e6 / 1e12
    assert top["peak"] == pytest.approx(alu)
    flops = m ** 3 / 3 + 2 * L * m * m + 2 * m ** 3 / 3
    assert top["achieved"] == pytest.approx(flops / 0.049e-3 / 1e12)
    assert top["frac"] == pytest.approx(top["achieved"] / alu)
    # an HBM phase: bytes of the 16-bit basis rows, hat priors and seed labels over its time
    pr = table["project"]
    assert pr["bound"] == "hbm" and pr["unit"] == "GB/s"
    assert pr["achieved"] == pytest.approx(N * (2 * m + 4 * lp + 4) / 0.024e-3 / 1e9)
    assert pr["frac"] == pytest.approx(pr["achieved"] / 6774.0)
    with pytest.raises(KeyError):
        bench.phase_work("nope", N, m, lp, S, L, steps)
