"""Compile-time resource checks of the hot kernels (no GPU needed).

The pass, recompute, reverse-step and gap kernels keep each thread's pixels in
registers or shared memory; a local-memory frame beyond the register spills
means a struct or array was placed in local memory (a runtime-indexed
parameter array or descriptor copy did exactly that to the batched list
kernels once, costing a fifth of their throughput). ptxas reports the frame
and spill sizes of every kernel it compiles."""
import os
import re
import subprocess
from concurrent.futures import ThreadPoolExecutor

import pytest

from paper_2109_05496_gb300 import build

UNITS = ("plan.cu", "plan_list_tv1.cu", "pass_tv1.cu", "pass_gap_tv1.cu", "backward.cu", "denoise.cu")
KERNELS = ("fgp_pass_kernel", "fgp_pass_list_kernel", "fgp_hist_pass_kernel", "adj_stream_kernel",
           "adj2_stream_kernel", "fgp_gap_kernel", "fgp_gap_list_kernel", "fgp_finalize_kernel",
           "fgp_gap_finish_kernel")


def _ptxas_report(unit, out_dir):
    src = os.path.join(build.CSRC, unit)
    cmd = [build.nvcc()] + build.ARCH + build.CFLAGS + ["-Xptxas", "-v", "-c", src, "-o",
                                                        os.path.join(out_dir, unit + ".o")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    return r.stderr


def _frames(report):
    """(mangled name, stack frame bytes, spill store bytes) per compiled kernel."""
    out = []
    lines = report.splitlines()
    for i, ln in enumerate(lines):
        m = re.search(r"Function properties for (\S+)", ln)
        if not m or i + 1 >= len(lines):
            continue
        f = re.search(r"(\d+) bytes stack frame, (\d+) bytes spill stores", lines[i + 1])
        if f:
            out.append((m.group(1), int(f.group(1)), int(f.group(2))))
    return out


@pytest.fixture(scope="module")
def reports(tmp_path_factory):
    try:
        build.nvcc()
    except RuntimeError:
        pytest.skip("nvcc not available")
    d = str(tmp_path_factory.mktemp("ptxas"))
    with ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        return dict(zip(UNITS, ex.map(lambda u: _ptxas_report(u, d), UNITS)))


def test_hot_kernels_have_no_local_arrays(reports):
    seen = 0
    for unit, rep in reports.items():
        for name, frame, spill in _frames(rep):
            if not any(k in name for k in KERNELS):
                continue
            seen += 1
            # a frame is allowed only for register spills (rounded to 8-byte slots)
            assert frame <= ((spill + 7) // 8) * 8 + 8, (unit, name, frame, spill)
    assert seen >= 64   # every TV type / constraint / configuration instantiation was checked


def test_default_pass_fits_two_blocks_per_sm(reports):
    # config 11 (T = 4, 64 x 32, 512 threads) needs <= 64 registers for two
    # resident blocks per SM, and no spills in the specialisations of the
    # benchmarked constraints (none, amplitude bound, support rectangle; the
    # general mask / box one may spill a little)
    rep = reports["pass_tv1.cu"]
    lines = rep.splitlines()
    found = 0
    for i, ln in enumerate(lines):
        m = re.search(r"Function properties for _ZN3ctv15fgp_pass_kernelILi1ELi1ELi4ELi2ELi8ELi4ELi(\d)E", ln)
        if not m:
            continue
        found += 1
        if int(m.group(1)) < 3:
            assert "0 bytes spill stores" in lines[i + 1], lines[i + 1]
        regs = re.search(r"Used (\d+) registers", lines[i + 2])
        assert regs and int(regs.group(1)) <= 64, lines[i + 2]
    assert found == 4   # the four constraint specialisations


def test_large_image_default_fits_one_block_per_sm(reports):
    # config 18 (T = 8, 64 x 64, 1024 threads, the large-image default with a support
    # rectangle) must fit 64 registers per thread for its 1024-thread block, without
    # spills in the none / amplitude / rectangle specialisations
    rep = reports["pass_tv1.cu"]
    lines = rep.splitlines()
    found = 0
    for i, ln in enumerate(lines):
        m = re.search(r"Function properties for _ZN3ctv15fgp_pass_kernelILi1ELi1ELi8ELi2ELi16ELi4ELi(\d)E", ln)
        if not m:
            continue
        found += 1
        if int(m.group(1)) < 3:
            assert "0 bytes spill stores" in lines[i + 1], lines[i + 1]
        regs = re.search(r"Used (\d+) registers", lines[i + 2])
        assert regs and int(regs.group(1)) <= 64, lines[i + 2]
    assert found == 4
