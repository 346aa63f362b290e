"""Failure detection on the GPU without a fault: every mbarrier wait of the
tensor-core fitness kernels is bounded.  With the handle's wait budget cut
to a few SM clock ticks (mgfwa_debug_wait_budget) an ordinary wait runs out
-- no arrival is withheld, nothing faults -- and the kernel aborts: every
role leaves its loop, drains its own copies and MMAs, frees TMEM and
returns, and the call reports MGFWA_ETIMEOUT.  The handle then works again
with the default budget (bitwise the same fitness as before), and a new
handle on the same device evaluates too, so TMEM was released.  Both
tensor-core kernels: the CTA-pair kernel (784-64-10) and the one-CTA kernel
(a three-layer net)."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build()
    import paper_2501_03944_gb300 as p
    return p


@pytest.mark.parametrize("widths,acts", [((784, 64, 10), (1,)), ((64, 64, 32, 5), (1, 0))])
def test_bounded_wait_gives_up_and_the_handle_recovers(pkg, widths, acts):
    w = W.scaled(W.MLP_784_64_10, widths=widths, acts=acts, n_samples=300, n_fireworks=2, sparks_per_firework=12,
                 guiding_per_firework=2)
    X, y = W.make_data(w)
    xs = W.random_vectors(24, w.dim, -1.0, 1.0, seed=9)
    with pkg.Mgfwa.for_workload(w, 3, precision=pkg.MGFWA_BF16, X=X, y=y) as run:
        ref = run.evaluate(xs, pkg.MGFWA_BF16)
        run.wait_budget(16)
        with pytest.raises(pkg.MgfwaError) as e:
            run.evaluate(xs, pkg.MGFWA_BF16)
        assert e.value.status == pkg.MGFWA_ETIMEOUT
        assert "bounded device wait" in pkg.mgfwa_last_error(run.handle)
        run.wait_budget(0)
        again = run.evaluate(xs, pkg.MGFWA_BF16)
        assert np.array_equal(again, ref)
        assert run.step(2) == pkg.MGFWA_OK
    with pkg.Mgfwa.for_workload(w, 3, precision=pkg.MGFWA_BF16, X=X, y=y) as run2:
        assert np.array_equal(run2.evaluate(xs, pkg.MGFWA_BF16), ref)
