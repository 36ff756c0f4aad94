"""Resource budget of the persistent sweeps, from the compiler's own report
(nvcc -Xptxas -v, no GPU): four 256-thread blocks of k_sweep must fit on an
SM, so it may use at most 64 registers a thread; k_power (the all-green
sweep) runs three blocks an SM (the registers that hold the next warp
tile's bounds and sources), so it may use at most 85. Both keep their
shared memory static, within 48 KB a block, and the FP32 (MIXED) unit-weight
instantiations, those of the timed path, must not spill."""
import os
import re
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2008_02710_gb300", "csrc")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")


@pytest.fixture(scope="module")
def ptxas_report():
    if not os.path.exists(NVCC) and not shutil.which("nvcc"):
        pytest.skip("nvcc not available")
    nvcc = NVCC if os.path.exists(NVCC) else shutil.which("nvcc")
    with tempfile.TemporaryDirectory() as d:
        out = os.path.join(d, "sweep.o")
        r = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                            "-Xptxas", "-v", "-c", "-I", os.path.join(ROOT, "include"), "-o", out,
                            os.path.join(CSRC, "rlgl.cu")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    return r.stderr


def _entries(report, prefix):
    """(mangled name, registers, spill stores, static smem) of each entry
    function whose mangled name starts with prefix."""
    out = []
    lines = report.splitlines()
    for k, line in enumerate(lines):
        m = re.search(r"Compiling entry function '(%s[^']*)'" % re.escape(prefix), line)
        if not m:
            continue
        spill = regs = smem = None
        for nxt in lines[k + 1:k + 6]:
            s = re.search(r"(\d+) bytes spill stores", nxt)
            if s:
                spill = int(s.group(1))
            u = re.search(r"Used (\d+) registers.*?(\d+) bytes smem", nxt)
            if u:
                regs, smem = int(u.group(1)), int(u.group(2))
                break
        out.append((m.group(1), regs, spill, smem))
    return out


def test_sweep_fits_four_blocks_per_sm(ptxas_report):
    ent = _entries(ptxas_report, "_ZN4rlgl7k_sweep")
    assert len(ent) == 4  # {float, double} x {weighted, unit weights}
    for name, regs, spill, smem in ent:
        assert regs is not None and regs <= 64, (name, regs)
        assert smem is not None and smem <= 48 * 1024, (name, smem)


def test_mixed_sweep_does_not_spill(ptxas_report):
    ent = [e for e in _entries(ptxas_report, "_ZN4rlgl7k_sweepIf")]
    assert len(ent) == 2
    for name, regs, spill, smem in ent:
        assert spill == 0, (name, spill)


def test_power_sweep_fits_three_blocks_per_sm(ptxas_report):
    ent = _entries(ptxas_report, "_ZN4rlgl7k_power")
    assert len(ent) == 4
    for name, regs, spill, smem in ent:
        assert regs is not None and regs <= 85, (name, regs)
        assert smem is not None and 3 * smem <= 227 * 1024 and smem <= 48 * 1024, (name, smem)
    for name, regs, spill, smem in ent:
        # the unit-weight FP32 instantiation (the timed all-green path) does
        # not spill; the weighted one may spill a few words
        if name.startswith("_ZN4rlgl7k_powerIfLb0"):
            assert spill == 0, (name, spill)
        elif name.startswith("_ZN4rlgl7k_powerIf"):
            assert spill <= 64, (name, spill)
