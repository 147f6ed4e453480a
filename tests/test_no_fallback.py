"""The product path has no CPU fallback (CPU tests).

* Without libdirac.so the binding refuses to import.
* Without a CUDA device every simulation fails at creation with a CUDA error
  status, from Python and from a plain C client linked against the library;
  nothing is computed on the host.
"""
import ctypes as C
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def has_device():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def test_binding_refuses_to_import_without_the_library(tmp_path):
    pkg = tmp_path / "paper_1309_3452_gb300"
    shutil.copytree(os.path.join(ROOT, "paper_1309_3452_gb300"), str(pkg),
                    ignore=shutil.ignore_patterns("*.so", "csrc", "__pycache__", "_build"))
    r = subprocess.run([sys.executable, "-c", "import paper_1309_3452_gb300.dirac"], cwd=str(tmp_path),
                       capture_output=True, text=True, timeout=300)
    assert r.returncode != 0
    assert "ImportError" in r.stderr and "libdirac.so not found" in r.stderr


@pytest.mark.skipif(has_device(), reason="a CUDA device is present: the GPU tests cover this path")
def test_no_device_means_an_error_not_a_fallback():
    from paper_1309_3452_gb300 import build as B
    B.build()
    from paper_1309_3452_gb300 import dirac as D
    from paper_1309_3452_gb300 import workloads as W
    prob = W.Problem(2, (16, 16, 1), (1.0, 1.0, 1.0), 0.5, 0.1)
    for prec in (D.FP32, D.FP64):
        with pytest.raises(D.DiracError) as e:
            D.Sim(prob, prec)
        assert e.value.status == D.ERR_CUDA


@pytest.mark.skipif(has_device(), reason="a CUDA device is present: the GPU tests cover this path")
def test_c_client_without_device(tmp_path):
    from paper_1309_3452_gb300 import build as B
    lib = B.build()
    src = tmp_path / "client.c"
    src.write_text(r"""
#include <stdio.h>
#include "dirac.h"
int main(void) {
  dirac_fields f;
  dirac_fields_default(&f);
  f.V0 = 0.1;
  int N[3] = {16, 16, 1};
  double dx[3] = {1.0, 1.0, 1.0};
  dirac_sim* sim = 0;
  dirac_status st = dirac_create(&sim, 2, N, dx, 0.5, 0.1, &f, DIRAC_FP32, 0u, 0);
  printf("%d %d %s\n", (int)st, sim == 0, dirac_last_error(0));
  return 0;
}
""")
    exe = tmp_path / "client"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                    "-L", os.path.dirname(lib), "-ldirac", "-Wl,-rpath," + os.path.dirname(lib)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True, timeout=120).stdout.split(" ", 2)
    from paper_1309_3452_gb300 import dirac as D
    assert int(out[0]) == D.ERR_CUDA and out[1] == "1" and "cudaMalloc" in out[2]
