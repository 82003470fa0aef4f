"""Register use of the newest kernel forms, from ptxas's own report (nvcc
-Xptxas -v, sm_103a; no GPU needed): none spills to local memory, and each
fits the register budget its launch shape allows."""
import os
import re
import shutil
import subprocess

import pytest

KDIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_1904_08555_b300", "csrc", "kernels")

SRC = r"""
#include "ltimes.cuh"
#include "mass.cuh"
#include "update_chain.cuh"
namespace cj {
// LTimes on tcgen05, operands in tensor memory: the FP32 default tile (6 boxes, 4 stages, 4 converters)
template __global__ void ltimes_tc<36, 96, 0, 0, 1, 128, 4, 4, 0, 6, 0, 0, 1>(
    const float*, const float*, float*, long long, long long, const __grid_constant__ cj_tmap);
// and with 8 converter warps and a g-fastest input
template __global__ void ltimes_tc<36, 96, 1, 0, 8, 16, 4, 8, 0, 6, 0, 0, 1>(
    const float*, const float*, float*, long long, long long, const __grid_constant__ cj_tmap);
// FP32 update chain, 4 x 8 register blocks
template __global__ void update_chain<float, 64, 0, 8, 1>(const float*, float*, long long, int, double, int);
template __global__ void update_chain<float, 33, 1, 8, 3>(const float*, float*, long long, int, double, int);
// mass operator, one thread per 2-D element
template __global__ void mass_apply_thread<float, 5, 8, 128>(const float*, const float*, const float*, float*,
                                                               long long);
template __global__ void mass_apply_thread<double, 4, 6, 128>(const double*, const double*, const double*, double*,
                                                                long long);
}
"""

# function name fragment -> largest register count its launch allows
BUDGET = {
    "ltimes_tcILi36ELi96ELi0ELi0ELi1ELi128ELi4ELi4E": 168,   # 10 warps: ceil(10/4) = 3 per sub-partition
    "ltimes_tcILi36ELi96ELi1ELi0ELi8ELi16ELi4ELi8E": 128,    # 14 warps: 4 per sub-partition
    "update_chainIfLi64ELi0ELi8ELi1E": 128,
    "update_chainIfLi33ELi1ELi8ELi3E": 128,
    "mass_apply_threadIfLi5ELi8ELi128E": 255,
    "mass_apply_threadIdLi4ELi6ELi128E": 255,
}


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="nvcc not available")
def test_new_kernel_forms_do_not_spill(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    src = tmp_path / "forms.cu"
    src.write_text(SRC)
    r = subprocess.run([nvcc, "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-Xptxas", "-v",
                        "-I", KDIR, "-c", str(src), "-o", str(tmp_path / "forms.o")],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    report = {}
    current = None
    for line in r.stderr.splitlines():
        m = re.search(r"Compiling entry function '([^']+)'", line)
        if m:
            current = m.group(1)
            continue
        if current is None:
            continue
        m = re.search(r"(\d+) bytes spill stores, (\d+) bytes spill loads", line)
        if m:
            report.setdefault(current, {})["spills"] = int(m.group(1)) + int(m.group(2))
        m = re.search(r"Used (\d+) registers", line)
        if m:
            report.setdefault(current, {})["regs"] = int(m.group(1))
    for frag, budget in BUDGET.items():
        hits = [v for k, v in report.items() if frag in k]
        assert len(hits) == 1, (frag, list(report))
        assert hits[0]["spills"] == 0, (frag, hits[0])
        assert 0 < hits[0]["regs"] <= budget, (frag, hits[0])
