"""The symbolic front end (expression graph, reduce, df, code generation)
on the CPU: hash-consing and simplification rules of Sec. 2.1, derivatives
checked against the oracle's hand-derived partials (an independent
derivation), generated source compiling with NVRTC for sm_103a."""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
import paper_2508_15967_gb300 as gf
from paper_2508_15967_gb300 import symbolic as S
from paper_2508_15967_gb300 import workloads as W


def test_identical_subgraphs_are_built_once():
    x0, x1, _ = S.x()
    a = S.exp((x0 - 0.3) ** 2 * -2.0) * x1
    n = S.cache_size()
    b = S.exp((x0 - 0.3) ** 2 * -2.0) * x1
    assert a is b and S.cache_size() == n
    assert (x0 + x1) is (x1 + x0) and (x0 * x1) is (x1 * x0)


def test_reduce_rules():
    x0, x1, _ = S.x()
    assert (x0 + 0.0) is x0 and (0.0 + x0) is x0
    assert (x0 * 1.0) is x0 and (x0 * 0.0) is S.ZERO
    assert (S.const(2.0) * 3.0 + 1.0).value == 7.0
    assert (2.0 * x0 + 3.0 * x0) is (5.0 * x0)
    assert (x0 - x0) is S.ZERO
    assert (-(-x1)) is x1
    assert ((-x0) * (-x1)) is (x0 * x1)
    assert (x0 * x0) is x0 ** 2 and (x0 ** 2) ** 3 is x0 ** 6
    assert S.exp(S.ZERO) is S.ONE
    assert S.where_nonpos(S.const(-1.0), x0, x1) is x0


def test_df_rules():
    x0, x1, _ = S.x()
    assert S.df(x0 ** 3, "x0") is 3.0 * x0 ** 2
    assert S.df(S.const(4.0), "x0") is S.ZERO
    assert S.df(x1, "x0") is S.ZERO and S.df(x0, "x0") is S.ONE
    e = S.exp(2.0 * x0)
    assert S.df(e, "x0") is 2.0 * e
    assert S.df(10.0 * x0 + 0.5, "x0").value == 10.0


@pytest.mark.parametrize("kind", ["grin", "luneburg", "adjoint"])
def test_symbolic_gradients_match_the_oracle(kind):
    """D and its seven partials from the graph equal the oracle's
    hand-derived dispersion and gradients (two independent derivations)."""
    if kind == "grin":
        wl = W.grin(n=1)
        D = S.isotropic(S.grin_n2(1.5, 2.0) + S.gaussian_blobs(wl.medium["blobs"]))
        spec = wl.medium
        pts = np.random.default_rng(0).uniform(-0.3, 0.3, (40, 3))
    elif kind == "luneburg":
        D = S.isotropic(S.luneburg_n2())
        spec = dict(kind="luneburg")
        pts = np.random.default_rng(1).uniform(-1.2, 1.2, (40, 3))
    else:
        wl = W.adjoint(n=1)
        D = S.isotropic(S.luneburg_n2() + S.gaussian_blobs(wl.medium["blobs"]))
        spec = wl.medium
        pts = np.random.default_rng(2).uniform(-1.2, 1.2, (40, 3))
    k = np.random.default_rng(3).uniform(-1.5, 1.5, (40, 3))
    w = 1.3
    env = dict(x0=pts[:, 0], x1=pts[:, 1], x2=pts[:, 2], k0=k[:, 0], k1=k[:, 1], k2=k[:, 2],
               w=np.full(40, w))
    got = np.stack(S.evaluate(S.gradients(D), env), axis=1)
    ref = O.eval_dispersion(O.medium(**spec), pts, k, w)
    np.testing.assert_allclose(got[:, 0], ref[:, 0], rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(got[:, 1:4], ref[:, 1:4], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(got[:, 4:7], ref[:, 4:7], rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(got[:, 7], ref[:, 7], rtol=1e-13, atol=1e-13)


def test_generated_source_compiles_for_sm103a():
    wl = W.grin(n=1)
    D = S.isotropic(S.grin_n2(1.5, 2.0) + S.gaussian_blobs(wl.medium["blobs"]))
    src = S.medium_source(D)
    assert src.count("exp(") == 16                    # each blob's exponential emitted once
    st, log = gf.gf_jit_compile_check(src, "sm_103a")
    assert st == gf.GF_OK, log
    st, log = gf.gf_jit_compile_check(src.replace("out[7]", "out[7] = undefined_name;//"), "sm_103a")
    assert st == gf.GF_ERR_INVALID_ARG and "undefined_name" in log
