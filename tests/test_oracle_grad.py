"""Pins of the oracle's hand-derived adjoint.

* dot-product tests <J v, w> = <v, J^H w> for each linear stage (Fresnel
  propagation, far field, Fourier shift, chunk extraction, rotation);
* brute-force central finite differences of the oracle's loss over EVERY
  coordinate of delta, beta, the probe (real and imaginary parts) and the
  positions / hologram shifts on 8x8 problems: far field (LSQ and Poisson,
  two probe modes, a patch that leaves the volume), ptychotomography through
  the rotation, and near-field multi-distance holography;
* the zero-residual case: LSQ loss and all gradients vanish when the
  measured intensities equal the prediction.
"""
import math

import numpy as np
import pytest

from oracle import model


def _cplx(g, shape):
    return g.standard_normal(shape) + 1j * g.standard_normal(shape)


def test_dot_products_of_linear_stages():
    g = np.random.default_rng(0)
    N = 12
    u, w = _cplx(g, (N, N)), _cplx(g, (N, N))
    H = model.fresnel_kernel(N, 0.8)
    assert abs(np.vdot(w, model.propagate(u, H)) - np.vdot(model.propagate_T(w, H), u)) < 1e-10
    assert abs(np.vdot(w, model.farfield(u)) - np.vdot(model.farfield_T(w), u)) < 1e-10
    vol = g.standard_normal((3, 20, 20)); ch = g.standard_normal((3, N, N))
    for p0 in ([2, 3], [-4, 15], [30, 30]):
        gv = np.zeros_like(vol); model.put_chunk_T(gv, p0, ch)
        assert abs(np.sum(ch * model.take_chunk(vol, p0, N)) - np.sum(gv * vol)) < 1e-10
    v3, w3 = g.standard_normal((10, 3, 11)), g.standard_normal((10, 3, 11))
    for th in (0.3, 1.2, 2.9, np.pi / 4, 3 * np.pi / 4, -0.5):   # incl. the diagonal tilts
        assert abs(np.sum(w3 * model.rotate(v3, th)) - np.sum(model.rotate_T(w3, th) * v3)) < 1e-10


def _fd_check(pb, delta, beta, probe, pos, Im, tol=2e-6):
    L0, gd, gb, gp, gpos = model.loss_grad(pb, delta, beta, probe, pos, Im)
    f = lambda d, b, p, q: model.loss(pb, d, b, p, q, Im)
    assert abs(L0 - f(delta, beta, probe, pos)) <= 1e-14 * abs(L0) + 1e-300

    def central(get, put, x0):
        h = 1e-6 * max(1.0, abs(x0))
        put(x0 + h); fp = f(*state)
        put(x0 - h); fm = f(*state)
        put(x0)
        return (fp - fm) / (2 * h)

    state = [delta.copy(), beta.copy(), probe.copy(), pos.copy()]
    fds = {"delta": np.zeros_like(delta), "beta": np.zeros_like(beta),
           "probe": np.zeros_like(probe), "pos": np.zeros_like(pos)}
    for k, arr_i in (("delta", 0), ("beta", 1)):
        arr = state[arr_i]
        for idx in np.ndindex(arr.shape):
            def put(v, arr=arr, idx=idx): arr[idx] = v
            fds[k][idx] = central(None, put, arr[idx])
    P = state[2]
    for idx in np.ndindex(P.shape):
        def put_re(v, idx=idx): P[idx] = v + 1j * P[idx].imag
        def put_im(v, idx=idx): P[idx] = P[idx].real + 1j * v
        re = central(None, put_re, P[idx].real)
        im = central(None, put_im, P[idx].imag)
        fds["probe"][idx] = re + 1j * im
    Q = state[3]
    for idx in np.ndindex(Q.shape):
        def put(v, idx=idx): Q[idx] = v
        fds["pos"][idx] = central(None, put, Q[idx])
    for name, got in (("delta", gd), ("beta", gb), ("probe", gp), ("pos", gpos)):
        ref = fds[name]
        err = np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300)
        assert err < tol, (name, err)
    return L0


def _far_problem(loss, **kw):
    p = dict(N=8, L=3, M=2, B=3, Lz=3, Ly=12, Lx=12, kdz=253.354, lambda_dz_over_px2=0.4,
             farfield=1, nf=[], loss=loss, eps=1e-6, tomo=0, theta=0.0)
    p.update(kw)
    return model.Problem.of(p)


@pytest.mark.parametrize("loss", ["lsq", "poisson"])
def test_farfield_gradients_brute_force(loss):
    pb = _far_problem(loss)
    g = np.random.default_rng(11)
    delta = g.uniform(0, 1e-3, (pb.Lz, pb.Ly, pb.Lx)); beta = g.uniform(0, 2e-4, delta.shape)
    probe = _cplx(g, (pb.M, pb.N, pb.N)) * 3.0
    pos = np.array([[1.2, 2.7], [-3.3, 5.8], [4.35, 1.1]])     # second patch leaves the volume
    Im = model.forward(pb, delta * 1.3, beta * 0.7, probe * 1.1, pos + 0.2)
    Im = np.random.default_rng(12).poisson(Im).astype(float)
    _fd_check(pb, delta, beta, probe, pos, Im)


def test_tomo_gradients_brute_force():
    pb = _far_problem("lsq", Lz=9, Ly=10, Lx=9, L=9, M=1, B=2, tomo=1, theta=0.45)
    g = np.random.default_rng(13)
    delta = g.uniform(0, 1e-3, (pb.Lz, pb.Ly, pb.Lx)); beta = g.uniform(0, 2e-4, delta.shape)
    probe = _cplx(g, (pb.M, pb.N, pb.N)) * 3.0
    pos = np.array([[1.2, 0.3], [0.4, 1.8]])
    Im = model.forward(pb, delta[::-1].copy(), beta, probe, pos)
    _fd_check(pb, delta, beta, probe, pos, Im)


def test_nearfield_gradients_brute_force():
    pb = model.Problem.of(dict(N=8, L=2, M=1, B=2, Lz=4, Ly=8, Lx=8, kdz=20.0, lambda_dz_over_px2=0.3,
                               farfield=0, nf=[0.05, 0.11], loss="lsq", eps=1e-6))
    g = np.random.default_rng(14)
    delta = g.uniform(0, 0.05, (pb.Lz, pb.Ly, pb.Lx)); beta = g.uniform(0, 0.002, delta.shape)
    probe = np.ones((1, 8, 8), complex) + 0.1 * _cplx(g, (1, 8, 8))
    shifts = np.array([[[1.3, -2.2], [0.4, 0.1]], [[-0.3, 3.35], [2.2, -1.4]]])
    Im = model.forward(pb, delta * 1.2, beta, probe, shifts + 0.25)
    _fd_check(pb, delta, beta, probe, shifts, Im)


def test_zero_residual_has_zero_loss_and_gradient():
    pb = _far_problem("lsq")
    g = np.random.default_rng(15)
    delta = g.uniform(0, 1e-3, (pb.Lz, pb.Ly, pb.Lx)); beta = g.uniform(0, 2e-4, delta.shape)
    probe = _cplx(g, (pb.M, pb.N, pb.N))
    pos = np.array([[1.2, 2.7], [3.3, 0.8], [2.35, 1.1]])
    Im = model.forward(pb, delta, beta, probe, pos)
    L, gd, gb, gp, gpos = model.loss_grad(pb, delta, beta, probe, pos, Im)
    assert L < 1e-25
    for a in (gd, gb, gp, gpos):
        assert np.max(np.abs(a)) < 1e-9


def test_nearfield_fresnel_number_gradient_brute_force():
    """dL/dN_F (free-propagation distance refinement) against central differences in N_F."""
    base = dict(N=8, L=1, M=1, B=2, Lz=2, Ly=8, Lx=8, kdz=20.0, lambda_dz_over_px2=0.0,
                farfield=0, nf=[0.05, 0.11, 0.3], loss="poisson", eps=1e-3)
    g = np.random.default_rng(17)
    delta = g.uniform(0, 0.05, (2, 8, 8)); beta = g.uniform(0, 0.002, delta.shape)
    probe = np.ones((1, 8, 8), complex)
    shifts = g.uniform(-2, 2, (2, 3, 2))
    Im = model.forward(model.Problem.of(base), delta * 1.2, beta, probe, shifts + 0.1)
    out = model.loss_grad(model.Problem.of(base), delta, beta, probe, shifts, Im, want_nf=True)
    for di in range(3):
        h = 1e-7
        pp = dict(base, nf=[v + (h if k == di else 0.0) for k, v in enumerate(base["nf"])])
        pm = dict(base, nf=[v - (h if k == di else 0.0) for k, v in enumerate(base["nf"])])
        # the loss is a mean over both problems; N_F is per problem in the gradient, shared here
        fd = (model.loss(model.Problem.of(pp), delta, beta, probe, shifts, Im)
              - model.loss(model.Problem.of(pm), delta, beta, probe, shifts, Im)) / (2 * h)
        assert abs(out[5][:, di].sum() - fd) <= 1e-6 * abs(fd) + 1e-12, (di, out[5][:, di].sum(), fd)


@pytest.mark.parametrize("far", [True, False])
def test_slice_gap_gradient_brute_force(far):
    """Sparse / variable multislice: dL/d(lambda dz_j / dx^2) against central differences."""
    if far:
        base = dict(N=8, L=4, M=2, B=2, Lz=4, Ly=12, Lx=12, kdz=253.354, lambda_dz_over_px2=0.0,
                    farfield=1, nf=[], loss="lsq", eps=1e-6, gaps=[0.4, 1.7, 0.9])
        pos = np.array([[1.2, 2.7], [3.3, 0.8]])
    else:
        base = dict(N=8, L=3, M=1, B=2, Lz=6, Ly=8, Lx=8, kdz=20.0, lambda_dz_over_px2=0.0,
                    farfield=0, nf=[0.05, 0.11], loss="poisson", eps=1e-3, gaps=[0.6, 2.2])
        pos = np.array([[[1.3, -2.2], [0.4, 0.1]], [[-0.3, 3.35], [2.2, -1.4]]])
    g = np.random.default_rng(19)
    shape = (base["Lz"], base["Ly"], base["Lx"])
    delta = g.uniform(0, 2e-3 if far else 0.05, shape); beta = g.uniform(0, 2e-4 if far else 0.002, shape)
    probe = _cplx(g, (base["M"], 8, 8)) * (3.0 if far else 0.1) + (0 if far else 1.0)
    pb = model.Problem.of(base)
    Im = model.forward(pb, delta * 1.2, beta, probe, pos + 0.1)
    out = model.loss_grad(pb, delta, beta, probe, pos, Im, want_gaps=True)
    gg = out[-1]
    for j in range(len(base["gaps"])):
        h = 1e-6
        gp = list(base["gaps"]); gp[j] += h
        gm = list(base["gaps"]); gm[j] -= h
        fd = (model.loss(model.Problem.of(dict(base, gaps=gp)), delta, beta, probe, pos, Im)
              - model.loss(model.Problem.of(dict(base, gaps=gm)), delta, beta, probe, pos, Im)) / (2 * h)
        assert abs(gg[j] - fd) <= 1e-6 * max(abs(fd), 1e-12) + 1e-13, (j, gg[j], fd)
    # uniform gaps reproduce the equal-spacing model
    pu = model.Problem.of(dict(base, gaps=[0.5] * len(base["gaps"])))
    pe = model.Problem.of(dict(base, gaps=None, lambda_dz_over_px2=0.5))
    np.testing.assert_allclose(model.forward(pu, delta, beta, probe, pos), model.forward(pe, delta, beta, probe, pos),
                               rtol=1e-13)


@pytest.mark.parametrize("tomo,loss", [(1, "lsq"), (0, "poisson")])
def test_position_offset_gradient_brute_force(tomo, loss):
    """Per-angle position offset (Sec. 2.3.2): central differences of the loss in one offset added
    to every position of the batch against offset_loss_grad."""
    if tomo:
        pb = _far_problem(loss, Lz=9, Ly=10, Lx=9, L=9, M=1, B=3, tomo=1, theta=0.45)
    else:
        pb = _far_problem(loss)
    g = np.random.default_rng(17)
    delta = g.uniform(0, 1e-3, (pb.Lz, pb.Ly, pb.Lx)); beta = g.uniform(0, 2e-4, delta.shape)
    probe = _cplx(g, (pb.M, pb.N, pb.N)) * 3.0
    pos = np.array([[1.2, 0.3], [0.4, 1.8], [2.1, -0.7]])[:pb.B]
    Im = model.forward(pb, delta * 1.2, beta, probe, pos + 0.15)
    L0, g_off = model.offset_loss_grad(pb, delta, beta, probe, pos, Im)
    h = 1e-6
    for a in range(2):
        e = np.zeros(2)
        e[a] = h
        fd = (model.loss(pb, delta, beta, probe, pos + e, Im) - model.loss(pb, delta, beta, probe, pos - e, Im)) / (2 * h)
        assert abs(fd - g_off[a]) <= 2e-6 * max(abs(fd), 1e-12) + 1e-12, (a, fd, g_off[a])
