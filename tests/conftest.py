import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: oracle test that takes more than a few seconds")


# ---------------------------------------------------------------------------
# Host programs built from the library's sources (the -m "not gpu" tests that
# check host-side set-up code against the oracle): each translation unit is
# compiled once per session and linked into the test's own driver.
# ---------------------------------------------------------------------------
import shutil  # noqa: E402
import subprocess  # noqa: E402

import pytest  # noqa: E402

CSRC = os.path.join(ROOT, "paper_2205_05840_gb300", "csrc")
NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17", "--expt-relaxed-constexpr", "-w",
              "-I", os.path.join(ROOT, "include"), "-I", CSRC]


@pytest.fixture(scope="session")
def host_build(tmp_path_factory):
    """build(driver_source, units) -> path of a host executable made of the
    driver and the named library translation units (objects cached for the
    session); skips the test when nvcc is missing."""
    nvcc = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    d = str(tmp_path_factory.mktemp("host_build"))
    objs: dict = {}
    count = [0]

    def obj(unit: str) -> str:
        if unit not in objs:
            o = os.path.join(d, unit + ".o")
            subprocess.run([nvcc, *NVCC_FLAGS, "-c", os.path.join(CSRC, unit), "-o", o], check=True,
                           capture_output=True)
            objs[unit] = o
        return objs[unit]

    def build(driver: str, units) -> str:
        count[0] += 1
        src = os.path.join(d, f"drv{count[0]}.cu")
        with open(src, "w") as fh:
            fh.write(driver)
        exe = os.path.join(d, f"drv{count[0]}")
        subprocess.run([nvcc, *NVCC_FLAGS, src, *[obj(u) for u in units], "-o", exe], check=True,
                       capture_output=True)
        return exe

    return build
