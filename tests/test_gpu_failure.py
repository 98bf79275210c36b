"""Failure detection without a GPU fault: the tensor-core kernels' completion waits are
bounded in time.  The library's self-test withholds the MMAs of one contraction, so its
barrier never fires; the kernel must give up, free its tensor memory and report, and the
same stream must then run a correct contraction."""
import time

import pytest

from paper_2409_05285_gb300 import binding

pytestmark = pytest.mark.gpu


def test_tensor_core_wait_runs_out_and_context_stays_usable():
    from paper_2409_05285_gb300.build import build
    build()
    lib = binding.load()
    t0 = time.time()
    rc = lib.peps_selftest_tc_timeout()
    dt = time.time() - t0
    assert rc == binding.PEPS_OK, rc
    assert dt >= 1.0   # the bounded waits (1 s each) did run out
    # a regular context on the same device still works afterwards
    ctx = binding.Context(4, 4, 2, 4, 8, precision=binding.PEPS_TF32, seed=1)
    la, sg, es, ea, _ = ctx.eval_batch(with_O=False)
    assert (sg != 0).all()
    ctx.close()
