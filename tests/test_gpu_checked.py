"""The checked build (-DRDHEI_CHECK) on the GPU: its kernels test every data-dependent
index (tile-map targets, slot-buffer and output-word positions) before the access and
report RDHEI_EBOUNDS instead of touching memory out of range.  A parity subset runs in
a child process that loads the checked library; every call must finish with status 0
(no check fired) and match the oracle byte for byte, as with the normal build."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# glide and MED variants, ragged and degenerate shapes, payload fractions, mixed batches
SUBSET = [
    ("tests/test_gpu_parity.py", "not c1_full_size"),
    ("tests/test_gpu_med.py", "shapes or edge or mixed or widths"),
    ("tests/test_gpu_configs.py", "uneven or mixed_variants"),
    ("tests/test_gpu_fused.py", "shapes or partial or equals_separable"),
    ("tests/test_zz_no_alloc.py", "twice or largest or side_stream"),
]


@pytest.fixture(scope="module")
def checked_env():
    from paper_2302_07992_gb300 import build
    build.build(checked=True)
    env = dict(os.environ, RDHEI_CHECKED="1")
    r = subprocess.run([sys.executable, "-c", "from paper_2302_07992_gb300 import rdhei; "
                        "assert rdhei.checked(), rdhei.LIBRARY; print(rdhei.LIBRARY)"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip().endswith("librdhei_check.so")
    return env


@pytest.mark.parametrize("path,select", SUBSET)
def test_parity_under_the_checked_build(checked_env, path, select):
    r = subprocess.run([sys.executable, "-m", "pytest", path, "-q", "-x", "-m", "gpu", "-k", select,
                        "-p", "no:cacheprovider"],
                       cwd=ROOT, env=checked_env, capture_output=True, text=True, timeout=1200)
    tail = "\n".join((r.stdout + r.stderr).splitlines()[-25:])
    assert r.returncode == 0, tail
    assert " passed" in r.stdout and "failed" not in r.stdout, tail
