"""Bounded device waits end with a status instead of hanging.

The sort kernels place a bin's merged entries after a decoupled look-back: a
bin waits, with a spin bound, until the bins before it have published their
counts.  A test build of the library makes that wait run out on purpose: its
sort kernels never take the first bin of their range, so the next bin's
predecessor never publishes, and its spin bound is short.  The call must
return, and the device status must read PB_ERR_TIMEOUT, for a single product
(warp look-back) and for a batch (block look-back).  The test build runs in a
child process so that it never shares a process with the product library.
"""
import os
import subprocess
import sys
import textwrap

import pytest
import torch

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2002_11302_gb300")
TEST_LIB = os.path.join(PKG, "_build_timeout", "libpbspgemm_timeout.so")
PB_ERR_TIMEOUT = 7


@pytest.fixture(scope="module")
def timeout_lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_11302_gb300 import build
    return build.build(lib=TEST_LIB, obj_dir=os.path.join(PKG, "_build_timeout"),
                       defines=("PB_SPIN_LIMIT=1024", "PB_TEST_SKIP_FIRST_BIN=1"))


def _child(lib: str, body: str) -> str:
    code = textwrap.dedent(f"""
        import os, sys
        sys.path.insert(0, {ROOT!r})
        import torch
        import synth
        from paper_2002_11302_gb300 import binding
        binding.load_library({lib!r})
    """) + textwrap.dedent(body)
    env = dict(os.environ, PB_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    return r.stdout.strip().splitlines()[-1]


def test_single_product_lookback_times_out(timeout_lib):
    out = _child(timeout_lib, """
        A, B = synth.er(1 << 14, 8, seed=5)
        Ad, Bd = binding.csc_to_device(A), binding.csr_to_device(B)
        plan = binding.symbolic(Ad, Bd)
        assert plan.nbins > 2
        C = binding.alloc_output(plan, rowptr64=True)
        binding.numeric(plan, Ad, Bd, C, plan.workspace())
        torch.cuda.synchronize()
        print(plan.status())
    """)
    assert int(out) == PB_ERR_TIMEOUT


def test_batch_lookback_times_out(timeout_lib):
    out = _child(timeout_lib, """
        probs = [synth.er(4096, 8, seed=11), synth.er(3000, 6, seed=12)]
        bt = binding.Batch([binding.csc_to_device(a) for a, _ in probs],
                           [binding.csr_to_device(b) for _, b in probs])
        bt.run()
        torch.cuda.synchronize()
        print(bt.status())
    """)
    assert int(out) == PB_ERR_TIMEOUT
