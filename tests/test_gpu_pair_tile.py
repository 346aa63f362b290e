"""The CTA-pair fitness kernel's tiles.  Each spark's fitness (Sec. 3.3: the
cross-entropy of the network its position encodes, over the batch) is one
column block of a contraction; the kernel has two tile shapes -- the logits
written into the spark's own accumulator columns once its activations are
packed (256 / h1 sparks a tile), or into columns of their own
(256 / (h1 + logit rows)) -- a pipeline of 2 .. the deepest that fits, and
the partial last K atom (d_in not a multiple of the atom) either as a stage
of its own or through the K-tail buffers (32-byte swizzled, one load per
MMA of it).  Each spark's columns hold its own sums, accumulated in the
same order in every shape, so every shape, depth and K-tail choice must
give bitwise the same fitness: the creation-time tuner that picks the
fastest changes no result.  Checked on whole runs (fireworks, best, the
last generation's explosion and guiding fitness) over the networks the
kernel has: h1 = 64 and 128, 16 and 32 logit rows, d_in ending on a K atom
or not (one, two and three K-tail MMAs, a last MMA half zero fill), BF16 and
E4M3 operands, and the three-layer 3072-128-64-10 network (whose tile is always
the shared shape: only the depth varies)."""
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


def _cases(pkg):
    base = W.scaled(W.MLP_784_64_10, n_samples=600, n_fireworks=3, sparks_per_firework=20, guiding_per_firework=4,
                    eval_budget=W.budget_for_generations(3, 20, 4, 4))
    return [
        ("784-64-10 bf16", base, pkg.MGFWA_BF16, {}),
        ("96-64-10 bf16", W.scaled(base, widths=(96, 64, 10), n_samples=700), pkg.MGFWA_BF16, {}),
        ("200-64-20 bf16", W.scaled(base, widths=(200, 64, 20)), pkg.MGFWA_BF16, {}),
        ("256-128-10 bf16", W.scaled(base, widths=(256, 128, 10), acts=(0,)), pkg.MGFWA_BF16, {}),
        ("784-64-10 fp8", base, pkg.MGFWA_FP8, {"elite_rescore": 0}),
        ("3072-128-64-10 bf16", W.scaled(base, widths=(3072, 128, 64, 10), acts=(1, 1), n_samples=300,
                                         sparks_per_firework=12), pkg.MGFWA_BF16, {}),
        ("3072-128-64-10 fp8", W.scaled(base, widths=(3072, 128, 64, 10), acts=(1, 0), n_samples=520,
                                        sparks_per_firework=12), pkg.MGFWA_FP8, {"elite_rescore": 0}),
        # three K-tail MMAs (48 of 64 BF16 / 80 of 128 E4M3 elements in the partial atom)
        ("176-64-20 bf16", W.scaled(base, widths=(176, 64, 20)), pkg.MGFWA_BF16, {}),
        ("208-64-10 fp8", W.scaled(base, widths=(208, 64, 10)), pkg.MGFWA_FP8, {"elite_rescore": 0}),
    ]


def _make(pkg, w, seed, prec, kw):
    X, y = W.make_data(w)
    return pkg.Mgfwa.for_workload(w, seed, precision=prec, X=X, y=y, **kw)


def _state(pkg, h):
    return (h.read(pkg.MGFWA_BUF_FW_F), h.read(pkg.MGFWA_BUF_FW_X), h.read(pkg.MGFWA_BUF_FIT_E),
            h.read(pkg.MGFWA_BUF_FIT_G), h.read(pkg.MGFWA_BUF_BEST_F), h.info().generations)


def _kt(w, prec, pkg):
    """The K-tail MMAs of the network's partial last atom (0: none, or no full atom before it)."""
    bk, ke = (128, 32) if prec == pkg.MGFWA_FP8 else (64, 16)
    rem = w.widths[0] % bk
    k = -(-rem // ke)
    return k if w.widths[0] >= bk and 1 <= k <= 3 else 0


def _tiles(w):
    """The tile shapes the kernel has for the network: (shared, separate or None)."""
    h1, C = w.widths[1], w.widths[-1]
    if len(w.widths) == 4:
        return 256 // h1, None
    nl = 16 if C <= 16 else 32
    return 256 // h1, 256 // (h1 + nl)


@pytest.mark.parametrize("i", range(9))
def test_every_tile_gives_the_same_run(pkg, i):
    name, w, prec, kw = _cases(pkg)[i]
    shared, separate = _tiles(w)
    kt = _kt(w, prec, pkg)
    with _make(pkg, w, 31 + i, prec, kw) as h:
        S0, st0, tuned, kt0 = h.pair_tile()
        assert tuned == 1 and S0 in (shared, separate) and st0 >= 2 and kt0 in (0, kt), (name, S0, st0, tuned, kt0)
        h.run()
        ref = _state(pkg, h)
    assert ref[-1] >= 2
    tried = []
    for S in (shared, separate) if separate else (shared,):
        for st in range(2, 9):
            fits = False
            for k_tail in (0, 1) if kt else (0,):
                with _make(pkg, w, 31 + i, prec, kw) as h:
                    try:
                        h.set_pair_tile(S, st, k_tail)
                    except pkg.MgfwaError as e:
                        assert e.status == pkg.MGFWA_EINVAL and (st > 2 or k_tail == 1), (name, S, st, k_tail, str(e))
                        continue
                    assert h.pair_tile() == (S, st, 0, kt if k_tail else 0)
                    h.run()
                    got = _state(pkg, h)
                for a, b in zip(ref[:-1], got[:-1]):
                    assert np.array_equal(a, b), (name, S, st, k_tail)
                assert got[-1] == ref[-1]
                tried.append((S, st, k_tail))
                fits = True
            if not fits:
                break
    assert len(tried) >= (3 if separate else 2), tried
    if kt:
        assert any(t[2] == 1 for t in tried), (name, tried)


def test_tile_settings_out_of_range(pkg):
    name, w, prec, kw = _cases(pkg)[0]
    shared, separate = _tiles(w)
    with _make(pkg, w, 5, prec, kw) as h:
        for S, st, k_tail in ((shared + 1, 2, -1), (separate, 1, -1), (shared, 9, -1), (0, 2, -1), (shared, 2, 2),
                              (shared, 2, -2)):
            with pytest.raises(pkg.MgfwaError) as e:
                h.set_pair_tile(S, st, k_tail)
            assert e.value.status == pkg.MGFWA_EINVAL
        # the handle is still usable and on its tuned tile
        assert h.pair_tile()[2] == 1
        h.step(1)
    # K-tail buffers for a network whose d_in ends on a whole atom
    w256 = _cases(pkg)[3][1]
    with _make(pkg, w256, 5, pkg.MGFWA_BF16, {}) as h:
        assert h.pair_tile()[3] == 0
        with pytest.raises(pkg.MgfwaError) as e:
            h.set_pair_tile(_tiles(w256)[0], 2, 1)
        assert e.value.status == pkg.MGFWA_EINVAL


def test_off_the_pair_kernel(pkg):
    w = W.scaled(W.MLP_784_64_10, n_samples=256, n_fireworks=2, sparks_per_firework=8, guiding_per_firework=2)
    with _make(pkg, w, 3, pkg.MGFWA_FP32, {}) as h:
        assert h.pair_tile() == (-1, -1, -1, -1)
        with pytest.raises(pkg.MgfwaError):
            h.set_pair_tile(4, 2)
