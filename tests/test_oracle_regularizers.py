"""Pins of the regularizer oracle (Table regularizers): closed forms and brute-force gradients."""
import numpy as np

from oracle import regularizers as R


def test_closed_forms():
    z, y, x = np.meshgrid(np.arange(3), np.arange(4), np.arange(5), indexing="ij")
    ramp = 2.0 * x + 0.5 * y - 1.0 * z           # forward differences 2, 0.5, -1 everywhere
    No = ramp.size
    tv = (2.0 * 3 * 4 * 4 + 0.5 * 3 * 3 * 5 + 1.0 * 2 * 4 * 5) / No
    r, _, _ = R.regularize(ramp, np.zeros_like(ramp), gamma_tv=1.0)
    assert abs(r - tv) < 1e-14
    c = np.full((2, 3, 4), -0.25)
    r, gd, gb = R.regularize(c, 2 * c, alpha_delta=3.0, alpha_beta=5.0, gamma_tv=7.0)
    assert abs(r - (3.0 * 0.25 + 5.0 * 0.5)) < 1e-14            # constant: no TV, mean |.|
    np.testing.assert_allclose(gd, -3.0 / c.size)
    np.testing.assert_allclose(gb, -5.0 / c.size)
    w = R.l1_weights(np.array([[[0.0, -2.0, 1.0]]]), 0.5)
    np.testing.assert_allclose(w.ravel(), [4.0, 0.8, 2.0 / 1.5])


def test_gradients_brute_force():
    g = np.random.default_rng(3)
    d = g.standard_normal((3, 4, 5))
    b = g.standard_normal((3, 4, 5))
    wd, wb = g.uniform(0.5, 2, d.shape), g.uniform(0.5, 2, b.shape)
    kw = dict(alpha_delta=0.7, alpha_beta=1.3, w_delta=wd, w_beta=wb, gamma_tv=0.9)
    r0, gd, gb = R.regularize(d, b, **kw)
    for arr, grad, which in ((d, gd, 0), (b, gb, 1)):
        fd = np.zeros_like(arr)
        for idx in np.ndindex(arr.shape):
            h = 1e-7
            a0 = arr[idx]
            arr[idx] = a0 + h
            rp = R.regularize(d, b, **kw)[0]
            arr[idx] = a0 - h
            rm = R.regularize(d, b, **kw)[0]
            arr[idx] = a0
            fd[idx] = (rp - rm) / (2 * h)
        assert np.max(np.abs(fd - grad)) < 1e-7, which
