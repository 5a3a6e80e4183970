"""The packed neighbour records the library builds on the host (specialised,
penalty-specialised and wide layouts) decode back to the instance they came
from: spin ids, fields, every coupling and its J (padding entries at the zero
row with J = 0), every copy link, link weights and penalty fields.  A small
C++ program (tests/_records_check.cpp) calls the library's preparation step on
random instances and decodes the records by the documented layouts.  No GPU."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_records_decode_to_the_instance(tmp_path):
    from paper_2506_14781_gb300 import build as b

    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    lib = b.build()
    cuda_inc = next((p for p in ("/usr/local/cuda/include",) if os.path.isdir(p)), None)
    if cuda_inc is None:
        pytest.skip("CUDA headers not available")
    exe = str(tmp_path / "records_check")
    cmd = [gxx, "-std=c++17", "-O1", f"-I{os.path.join(ROOT, 'include')}",
           f"-I{os.path.join(ROOT, 'paper_2506_14781_gb300', 'csrc')}", f"-I{cuda_inc}",
           os.path.join(ROOT, "tests", "_records_check.cpp"), lib, f"-Wl,-rpath,{os.path.dirname(lib)}",
           "-o", exe]
    subprocess.run(cmd, check=True, capture_output=True)
    res = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert res.returncode == 0 and res.stdout.startswith("ok"), res.stdout + res.stderr
