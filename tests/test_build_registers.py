"""Register budgets of the batched sweep kernels (CPU, nvcc only).

ptxas reports each kernel's stack frame and spill bytes. The marching kernels the tuner picks
and the FP64 xi tiles keep the spill figures their launch bounds were chosen for. A change that
pushes them into local memory fails here before it costs GPU time. Figures for WENOIU5-1MP,
the scheme the bench times.
"""
import concurrent.futures as cf
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_1810_11103_gb300", "csrc")

# (file, kernel name prefix of WENOIU5-1MP, spill-store bytes allowed)
BUDGETS = [
    ("batch_fp64.cu", "_ZN3fsp18march_batch_kernelILi2ELi0EddE", 0),
    ("batch_fp64.cu", "_ZN3fsp22march_eta_batch_kernelILi2ELi2EddE", 0),
    ("batch_fp64.cu", "_ZN3fsp18sweep_batch_kernelILi2ELi0ELi0EddLi2EE", 0),
    ("batch_fp32.cu", "_ZN3fsp18march_batch_kernelILi2ELi0EffE", 0),
    ("batch_fp32.cu", "_ZN3fsp22march_eta_batch_kernelILi2ELi2EffE", 0),
    # the RK stage that also takes the next stage's line maxima (8 bytes: the column maximum)
    ("batch_fp32.cu", "_ZN3fsp22march_eta_batch_kernelILi2ELi3EffE", 8),
    ("batch_fp64.cu", "_ZN3fsp22march_eta_batch_kernelILi2ELi3EddE", 0),
    ("batch_mixed.cu", "_ZN3fsp18march_batch_kernelILi2ELi0EfdE", 16),
    ("batch_mixed.cu", "_ZN3fsp22march_eta_batch_kernelILi2ELi2EfdE", 0),
]


def _ptxas(path, tmp):
    from paper_1810_11103_gb300 import build as B
    out = os.path.join(tmp, os.path.basename(path) + ".o")
    r = subprocess.run([B.nvcc(), *B.ARCH, *B.FLAGS, "-Xptxas=-v", "-c", path, "-o", out],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    spills, cur = {}, None
    for line in (r.stdout + r.stderr).splitlines():
        m = re.search(r"Compiling entry function '(\S+)'", line)
        if m:
            cur = m.group(1)
            continue
        m = re.search(r"(\d+) bytes spill stores", line)
        if m and cur:
            spills[cur] = int(m.group(1))
            cur = None
    return spills


def test_spill_budgets(tmp_path):
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc is needed")
    files = sorted({f for f, _, _ in BUDGETS})
    with cf.ThreadPoolExecutor(len(files)) as ex:
        found = dict(zip(files, ex.map(lambda f: _ptxas(os.path.join(SRC, f), str(tmp_path)), files)))
    for f, prefix, allowed in BUDGETS:
        hits = [v for k, v in found[f].items() if k.startswith(prefix)]
        assert hits, f"{prefix} not compiled in {f}"
        assert max(hits) <= allowed, (f, prefix, max(hits), allowed)
