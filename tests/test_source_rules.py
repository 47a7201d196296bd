"""Static checks of the CUDA sources (CPU): every wait a kernel spins on is bounded, no kernel
traps or asserts on the device, kernels with grid-wide barriers are launched cooperatively, and
the build targets sm_103a only."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1607_04174_gb300", "csrc")


def _sources():
    out = {}
    for f in sorted(os.listdir(CSRC)):
        if f.endswith((".cu", ".cuh")):
            out[f] = open(os.path.join(CSRC, f)).read()
    return out


def _strip_comments(text):
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return re.sub(r"//[^\n]*", "", text)


def test_mbarrier_waits_are_bounded():
    """The mbarrier polls are mbar_try_wait (solve.cu) and mbar_poll (tc_common.cuh, used by the
    tensor-core kernels); each has one caller, a bounded loop that gives up (setting a timeout
    status) after a fixed number of polls."""
    src = {f: _strip_comments(t) for f, t in _sources().items()}
    polls = [f for f, t in src.items() for _ in re.finditer(r"mbarrier\.try_wait", t)]
    assert sorted(polls) == ["solve.cu", "tc_common.cuh"]
    g = src["tc_common.cuh"]
    assert len(re.findall(r"\bmbar_poll\s*\(", g)) == 2
    i = g.index("bool mbar_wait_limited(")
    body = g[i:g.index("\n}\n", i)]
    assert "mbar_poll(" in body and "RW_DEV_TIMEOUT" in body and "return false;" in body
    assert re.search(r"it\s*<=\s*\(1\s*<<\s*\d+\)", body)
    uses = re.findall(r"\bmbar_try_wait\s*\(", src["solve.cu"])
    assert len(uses) == 2  # its definition and the call inside mbar_wait_bounded
    i = src["solve.cu"].index("void mbar_wait_bounded(")
    body = src["solve.cu"][i:src["solve.cu"].index("\n}\n", i)]
    assert "mbar_try_wait(" in body and "RW_DEV_TIMEOUT" in body and "return;" in body
    assert re.search(r"it\s*>\s*\(1\s*<<\s*\d+\)", body)


def test_flag_polls_are_bounded():
    """The one poll on a flag in global memory (the projection that starts once the adaptive
    choice has published m) runs at most kEarlyPolls times and then takes the ordinary grid
    dependency wait, which ends when its predecessor ends."""
    src = {f: _strip_comments(t) for f, t in _sources().items()}
    polls = [f for f, t in src.items() for _ in re.finditer(r"ld\.acquire", t)]
    assert polls == ["solve.cu"]
    t = src["solve.cu"]
    assert re.search(r"constexpr int kEarlyPolls = 1 << 16;", t)
    i = t.index("ld.acquire")
    loop = t[t.rindex("for (", 0, i):i]
    assert re.match(r"for \(int it = 0; it < kEarlyPolls; \+\+it\)", loop)
    tail = t[i:t.index("__syncthreads();", i) + 200]
    assert "if (s_m < 0) rw_grid_wait();" in tail


def test_no_device_traps_or_asserts():
    for f, t in _sources().items():
        t = _strip_comments(t)
        assert "__trap" not in t, f
        assert not re.search(r"(?<![A-Za-z_])assert\s*\(", t), f


def test_grid_barrier_kernels_launch_cooperatively():
    checked = set()
    for f, t in _sources().items():
        t = _strip_comments(t)
        for m in re.finditer(r"this_grid\(\)", t):
            head = t[:m.start()]
            k = head.rfind("__global__")
            name = re.search(r"\b(k_[a-z0-9_]+)\s*\(", head[k:]).group(1)
            assert re.search(r"cudaLaunchCooperativeKernel\(\(void\*\)\s*" + name + r"\b", t), \
                (f, name)
            checked.add(name)
    assert {"k_jacobi", "k_pcg"} <= checked, checked


def test_build_targets_sm_103a_only():
    from paper_1607_04174_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
