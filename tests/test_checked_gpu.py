"""The bounds-checked build (libtop_checked.so, compiled with TOP_CHECKED).

Every kernel of that build checks the index bases it derives (pack,
trajectory, segment, junction slot, work-list entry) against the sizes of the
arrays they address; a failed check sets a bit in the handle's error word, the
access is skipped and the call returns TOP_E_BOUNDS.  These tests build that
variant and run the GPU parity, resume, cluster, polytope, adaptive-rho,
gradient and no-allocation suites against it in a child process: every call
must return TOP_OK with the same results the suites demand of the regular
build, i.e. no derived index ever left its array on those inputs.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SUITES = ["test_parity_gpu.py", "test_cluster_gpu.py", "test_resume_gpu.py", "test_polytope_gpu.py",
          "test_adaptive_rho_gpu.py", "test_grad_gpu.py", "test_sample_timealloc_gpu.py", "test_zz_no_alloc.py"]


def _build_checked():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "paper_2507_10290_gb300", "build.py"), "--checked"],
                       cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    return r.stdout.strip().splitlines()[-1]


def test_checked_library_is_separate_and_selected_by_environment():
    """CPU-side: TOP_CHECKED selects libtop_checked.so, which the build script names."""
    from paper_2507_10290_gb300 import build as B
    assert B.LIB_CHECKED != B.LIB and B.BUILD_CHECKED != B.BUILD
    code = ("import os, sys; os.environ['TOP_CHECKED'] = '1'; sys.path.insert(0, %r); "
            "import importlib.util as u; spec = u.find_spec('paper_2507_10290_gb300.top'); "
            "src = open(spec.origin).read(); "
            "assert 'libtop_checked.so' in src and 'TOP_CHECKED' in src; print('ok')" % ROOT)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stderr


@pytest.mark.gpu
def test_parity_suites_under_the_checked_build():
    lib = _build_checked()
    assert lib.endswith("libtop_checked.so")
    env = dict(os.environ, TOP_CHECKED="1")
    probe = subprocess.run([sys.executable, "-c",
                            "from paper_2507_10290_gb300 import top; print(top.LIB_PATH)"],
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert probe.returncode == 0 and probe.stdout.strip().endswith("libtop_checked.so"), probe.stderr
    cmd = [sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider",
           "-k", "not full_size", *[os.path.join("tests", s) for s in SUITES]]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=2400)
    tail = (r.stdout[-3000:] + r.stderr[-2000:])
    assert r.returncode == 0, tail
    assert " passed" in r.stdout and "failed" not in r.stdout.splitlines()[-1], tail
