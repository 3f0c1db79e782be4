import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a GB300 and the CUDA library")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle


def golden_path(name):
    return os.path.join(ROOT, "tests", "golden", name)


def stdp_tables():
    """(ltp, ltd) lists indexed by lag 0..255 from the golden file."""
    ltp, ltd = [], []
    with open(golden_path("stdp_q16_tables.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, p, m = (int(x) for x in line.split())
            assert k == len(ltp)
            ltp.append(p)
            ltd.append(m)
    return ltp, ltd


def build_readme_c_example(tmp_path, lib_path):
    """Compile examples/readme_example.c (the smallest use of the C ABI)
    against include/snn.h and link it with the engine library at lib_path;
    returns the executable's path."""
    import subprocess
    src = os.path.join(ROOT, "examples", "readme_example.c")
    exe = tmp_path / "readme_example"
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                    "-o", str(exe), src, os.path.abspath(lib_path)], check=True)
    return exe
