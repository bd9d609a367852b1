"""The C-ABI used from plain C: tests/c_abi_example.c is compiled against
include/bicoptor.h and the library, run on the GPU, and must print "ok"."""
import os
import subprocess

import pytest

from paper_2309_04909_gb300 import _native
from tests._util import cuda_ok

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")]

HERE = os.path.dirname(os.path.abspath(__file__))


def test_plain_c_caller(tmp_path):
    lib = _native.build()
    exe = tmp_path / "c_abi_example"
    cuda = os.path.dirname(os.path.dirname(_native.nvcc()))
    subprocess.run(["gcc", "-O1", "-std=c11", "-I", _native.INCLUDE,
                    "-I", os.path.join(cuda, "include"), os.path.join(HERE, "c_abi_example.c"),
                    "-o", str(exe), os.path.abspath(lib), "-L", os.path.join(cuda, "lib64"),
                    "-lcudart", f"-Wl,-rpath,{os.path.dirname(os.path.abspath(lib))}",
                    f"-Wl,-rpath,{os.path.join(cuda, 'lib64')}"], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == "ok"
