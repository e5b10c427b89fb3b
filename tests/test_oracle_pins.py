"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these tests re-types the oracle's formulas: they use closed forms,
identities, brute force, Monte Carlo or finite differences, chosen so that a
dropped term, a wrong sign, a transposed operand or a wrong index in the
oracle fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_2405_20067_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def raw_from(oracle, mix, ch=None):
    arrs = [mix["mean"], mix["theta"], mix["alpha_raw"], mix["color_raw"]]
    if ch is None:
        arrs += [None] * 4
    else:
        arrs += [ch["u_theta"], ch["m_u"], ch["c_alpha_raw"], ch["c_color_raw"]]
    return oracle.Raw.from_arrays(arrs, has_children=ch is not None)


def lower_via_tanh(N, theta_row):
    """Covariance factor from raw values through the identities
    exp(ln s) = s on the diagonal and 2 sigmoid(t) - 1 = tanh(t / 2)."""
    L = np.zeros((N, N))
    k = 0
    for i in range(N):
        for j in range(i + 1):
            L[i, j] = math.exp(theta_row[k]) if i == j else math.tanh(theta_row[k] / 2.0)
            k += 1
    return L


def single(N, mean, theta, a=0.0, gam=(0.0, 0.0, 0.0)):
    return {"mean": np.asarray(mean, np.float64).reshape(1, N),
            "theta": np.asarray(theta, np.float64).reshape(1, -1),
            "alpha_raw": np.array([a], np.float64),
            "color_raw": np.asarray(gam, np.float64).reshape(1, 3)}


# ---- Eq. 1: values fixed by the definition --------------------------------

def test_value_at_mean_is_weight(oracle):
    """Eq. 1: G(0) = 1, so a query at the mean returns w exactly."""
    N = 6
    mix = synth.mixture(N, 5, seed=3)
    raw = raw_from(oracle, mix)
    L, m, w = oracle.activate(raw)
    for g in range(5):
        y = oracle.eval(L[g:g + 1], m[g:g + 1], w[g:g + 1], m[g:g + 1])
        assert np.array_equal(y[0], w[g])


def test_golden_closed_forms(oracle):
    """Eq. 1 with N = 1 and isotropic factors: exp(-d^2 / (2 sigma^2))."""
    with open(os.path.join(GOLDEN, "closed_forms.json")) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        N = c["N"]
        P = N * (N + 1) // 2
        theta = np.zeros(P)
        k = 0
        for i in range(N):
            for j in range(i + 1):
                if i == j:
                    theta[k] = math.log(c["sigma"])
                k += 1
        one = single(N, c["mean"], theta, a=math.log(c["alpha"]), gam=[0.0, 0.0, 0.0])
        raw = oracle.Raw.from_arrays([one["mean"], one["theta"], one["alpha_raw"],
                                      one["color_raw"], None, None, None, None], False)
        L, m, w = oracle.activate(raw)
        y = oracle.eval(L, m, w, np.asarray(c["x"], np.float64).reshape(1, N))
        # colour raw 0 -> sigmoid 1/2 on every channel
        expect = c["alpha"] * 0.5 * c["value"]
        np.testing.assert_allclose(y[0], expect, rtol=1e-14, err_msg=c["cite"])


def test_covariance_factor_semantics(oracle):
    """Section 3.1: L maps N(0, I) to the component, so at x = m + L xi the
    exponent is exactly |xi|^2 (L from the tanh identity, not the oracle)."""
    r = np.random.default_rng(5)
    N = 6
    mix = synth.mixture(N, 4, seed=9)
    raw = raw_from(oracle, mix)
    L, m, w = oracle.activate(raw)
    for g in range(4):
        Lt = lower_via_tanh(N, mix["theta"][g].astype(np.float64))
        np.testing.assert_allclose(L[g], Lt, rtol=1e-14, atol=1e-15)
        xi = r.normal(size=(50, N))
        x = m[g] + xi @ Lt.T
        y = oracle.eval(L[g:g + 1], m[g:g + 1], w[g:g + 1], x)
        expect = np.exp(-0.5 * np.sum(xi ** 2, axis=1))[:, None] * w[g]
        np.testing.assert_allclose(y, expect, rtol=1e-12)


def test_diagonal_closed_form(oracle):
    """Diagonal factor: exponent is sum_i (x_i - m_i)^2 / L_ii^2."""
    r = np.random.default_rng(1)
    N = 4
    sig = np.array([0.2, 0.5, 1.3, 0.07])
    P = N * (N + 1) // 2
    theta = np.full(P, 0.0)  # off-diagonals activate to 0
    k = 0
    for i in range(N):
        for j in range(i + 1):
            if i == j:
                theta[k] = math.log(sig[i])
            k += 1
    one = single(N, [0.1, -0.2, 0.3, 0.0], theta, a=0.3, gam=[1.0, -1.0, 0.5])
    raw = oracle.Raw.from_arrays([one[k] for k in ("mean", "theta", "alpha_raw", "color_raw")]
                                 + [None] * 4, False)
    L, m, w = oracle.activate(raw)
    x = r.uniform(-1, 1, size=(40, N))
    y = oracle.eval(L, m, w, x)
    e = np.exp(-0.5 * np.sum(((x - m[0]) / sig) ** 2, axis=1))
    wexp = math.exp(0.3) / (1.0 + np.exp(-np.array([1.0, -1.0, 0.5])))
    np.testing.assert_allclose(y, e[:, None] * wexp, rtol=1e-13)


def test_explicit_inverse_and_lifted_forms(oracle):
    """The triangular-solve exponent equals (x-m)^T (L L^T)^{-1} (x-m) with a
    library inverse, and the lifted quadratic x^T A x - 2 m^T A x + m^T A m."""
    r = np.random.default_rng(2)
    N = 10
    mix = synth.mixture(N, 6, seed=11)
    raw = raw_from(oracle, mix)
    L, m, w = oracle.activate(raw)
    x = r.uniform(-1, 1, size=(30, N))
    for g in range(6):
        A = np.linalg.inv(L[g] @ L[g].T)
        d = x - m[g]
        s1 = np.einsum("qi,ij,qj->q", d, A, d)
        s2 = (np.einsum("qi,ij,qj->q", x, A, x) - 2 * x @ (A @ m[g]) + m[g] @ A @ m[g])
        y = oracle.eval(L[g:g + 1], m[g:g + 1], w[g:g + 1], x)
        np.testing.assert_allclose(y, np.exp(-0.5 * s1)[:, None] * w[g], rtol=1e-10)
        np.testing.assert_allclose(s1, s2, rtol=1e-9, atol=1e-9)


def test_weight_activation_identities(oracle):
    """Eq. 8 context: alpha = exp(a) and c = sigmoid(gamma); for gamma = 0 the
    colour is 1/2, and sigmoid(g) + sigmoid(-g) = 1."""
    N = 2
    one = single(N, [0, 0], [0.0, 0.0, 0.0], a=math.log(3.0), gam=[0.0, 2.0, -2.0])
    raw = oracle.Raw.from_arrays([one[k] for k in ("mean", "theta", "alpha_raw", "color_raw")]
                                 + [None] * 4, False)
    _, _, w = oracle.activate(raw)
    assert abs(w[0, 0] - 1.5) < 1e-15
    assert abs(w[0, 1] + w[0, 2] - 3.0) < 1e-14


def test_normalisation_matches_monte_carlo(oracle):
    """Eq. 1-2: the unnormalised Gaussian integrates to
    (2 pi)^{N/2} det(L) = (2 pi)^{N/2} prod_i L_ii.  Importance sampling
    from N(m, 2V) with numpy's generator and density."""
    r = np.random.default_rng(7)
    for N in (1, 3, 6):
        mix = synth.mixture(N, 1, seed=20 + N)
        raw = raw_from(oracle, mix)
        L, m, w = oracle.activate(raw)
        n = 200_000
        S = np.sqrt(2.0) * L[0]
        xs = m[0] + r.normal(size=(n, N)) @ S.T
        V2 = S @ S.T
        d = xs - m[0]
        logp = (-0.5 * np.einsum("qi,ij,qj->q", d, np.linalg.inv(V2), d)
                - 0.5 * N * math.log(2 * math.pi) - 0.5 * math.log(np.linalg.det(V2)))
        y = oracle.eval(L, m, w, xs)[:, 0] / w[0, 0]
        vals = y / np.exp(logp)
        est, se = vals.mean(), vals.std() / math.sqrt(n)
        exact = (2 * math.pi) ** (N / 2) * float(np.prod(np.exp(mix["theta"][0][
            [i * (i + 1) // 2 + i for i in range(N)]].astype(np.float64))))
        assert abs(est - exact) < 5 * se + 1e-12, (N, est, exact, se)


# ---- Eq. 6-7: children ------------------------------------------------------

def test_identity_child_duplicates_parent(oracle):
    """Eq. 6-7 with U = I (raw 0) and m_u = 0: the child coincides with the
    parent, so the output is (w_p + w_c) G_p(x)."""
    r = np.random.default_rng(4)
    N, G = 6, 3
    mix = synth.mixture(N, G, seed=5)
    P = N * (N + 1) // 2
    ch = {"u_theta": np.zeros((G, P)), "m_u": np.zeros((G, N)),
          "c_alpha_raw": np.log(np.array([0.1, 0.2, 0.3])),
          "c_color_raw": r.normal(size=(G, 3))}
    raw = raw_from(oracle, mix, ch)
    L, m, w = oracle.activate(raw)
    x = r.uniform(-1, 1, size=(20, N))
    for g in range(G):
        yp = oracle.eval(L[g:g + 1], m[g:g + 1], w[g:g + 1], x)
        both = oracle.eval(L[[g, G + g]], m[[g, G + g]], w[[g, G + g]], x)
        np.testing.assert_allclose(both, yp / w[g] * (w[g] + w[G + g]), rtol=1e-14)


def test_child_is_parent_frame_transform(oracle):
    """Eq. 6-7: the child is N(L_p m_u + m_p, (L_p U)(L_p U)^T); at
    x = m_c + L_p U xi its exponent is |xi|^2 (factors from tanh identity)."""
    r = np.random.default_rng(8)
    N, G = 5, 2
    mix = synth.mixture(N, G, seed=6)
    ch = synth.children(N, G, seed=7)
    raw = raw_from(oracle, mix, ch)
    L, m, w = oracle.activate(raw)
    for g in range(G):
        Lp = lower_via_tanh(N, mix["theta"][g].astype(np.float64))
        U = lower_via_tanh(N, ch["u_theta"][g].astype(np.float64))
        mc = Lp @ ch["m_u"][g].astype(np.float64) + mix["mean"][g]
        xi = r.normal(size=(30, N))
        x = mc + xi @ (Lp @ U).T
        c = G + g
        y = oracle.eval(L[c:c + 1], m[c:c + 1], w[c:c + 1], x)
        np.testing.assert_allclose(y, np.exp(-0.5 * (xi ** 2).sum(1))[:, None] * w[c], rtol=1e-11)


# ---- Eq. 3-5: culling -------------------------------------------------------

def _cull_case(seed=0, N=6, G=64, Q=1024, k=8, wscale=1.0):
    mix = synth.mixture(N, G, seed=seed)
    x = synth.queries_box(N, Q, seed + 1)
    proj = synth.projections(N, k, seed + 2)
    return mix, x.astype(np.float64), proj


@pytest.mark.parametrize("cutoff,k_sigma", [(1.0 / 255.0, 3.0), (0.0, 3.0), (0.0, 2.0)])
def test_cull_sound_against_brute_force(oracle, cutoff, k_sigma):
    """Every (tile, Gaussian) pair the exact and the contract culls drop has,
    at every query of the tile, exponent s > k^2 (Cauchy-Schwarz bound of
    Eq. 3-5); with a cutoff every dropped contribution is below the cutoff."""
    tile = 64
    mix, x, proj = _cull_case()
    raw = raw_from(oracle, mix)
    L, m, w = oracle.activate(raw)
    keep = oracle.cull_exact(L, m, w, x, tile, proj, cutoff, k_sigma)
    offs, ids = oracle.cull_contract(L, m, w, x, tile, proj, cutoff, k_sigma, 64)
    T, Ge = keep.shape
    contract = np.zeros_like(keep)
    for t in range(T):
        contract[t, ids[offs[t]:offs[t + 1]]] = 1
    # the contract is conservative with respect to the exact test
    assert np.all(contract >= keep)
    assert 0 < keep.sum() < keep.size  # something is culled, something kept
    for g in range(Ge):
        A = np.linalg.inv(L[g] @ L[g].T)
        d = x - m[g]
        s = np.einsum("qi,ij,qj->q", d, A, d).reshape(T, tile)
        if cutoff > 0:
            contrib = w[g].max() * np.exp(-0.5 * s)
            assert np.all(contrib[keep[:, g] == 0] < cutoff)
            assert np.all(contrib[contract[:, g] == 0] < cutoff)
        else:
            assert np.all(s[keep[:, g] == 0] > k_sigma ** 2)


def test_cull_contract_tile_selection_matches_full_run(oracle):
    """The contract restricted to a set of tiles (any order, repeats allowed)
    returns exactly those tiles' lists of the full run: the per-projection
    ranges and the keys come from the whole query set either way."""
    tile = 64
    mix, x, proj = _cull_case(seed=3, Q=1000)  # ragged last tile
    raw = raw_from(oracle, mix)
    L, m, w = oracle.activate(raw)
    offs, ids = oracle.cull_contract(L, m, w, x, tile, proj, 1.0 / 255.0, 3.0, 64)
    T = offs.size - 1
    sel = np.array([T - 1, 0, 5, 5, 11], dtype=np.int64)
    so, si = oracle.cull_contract(L, m, w, x, tile, proj, 1.0 / 255.0, 3.0, 64, tiles=sel)
    assert so.size == sel.size + 1 and so[0] == 0
    for i, t in enumerate(sel):
        np.testing.assert_array_equal(si[so[i]:so[i + 1]], ids[offs[t]:offs[t + 1]])
    eo, ei = oracle.cull_contract(L, m, w, x, tile, proj, 1.0 / 255.0, 3.0, 64, tiles=[])
    assert eo.tolist() == [0] and ei.size == 0


def test_condition_reproduces_the_nd_gaussian(oracle):
    """Section 3.2 conditioning: each Gaussian restricted to the constant
    inputs xc equals wc exp(-1/2 (x_p - mu)^T (T^T T)^-1 (x_p - mu)) at every
    position (checked against the N-D evaluation of that Gaussian alone, with
    the 3 x 3 inverse taken by numpy), and a diagonal factor gives the closed
    form mu = m_p, T = diag(L_pp) (covariance diag(L_pp^2)),
    wc = w exp(-1/2 sum ((xc - m_c) / L_cc)^2)."""
    N = 6
    mix = synth.mixture(N, 40, seed=21)
    ch = synth.children(N, 40, 22, spread=0.2)
    L, m, w = oracle.activate(raw_from(oracle, mix, ch))
    r = np.random.default_rng(23)
    xc = r.uniform(-0.5, 0.5, size=N - 3)
    mu, T, wc = oracle.condition(L, m, w, xc)
    xp = r.uniform(-1.0, 1.0, size=(50, 3))
    x = np.concatenate([xp, np.repeat(xc[None, :], 50, axis=0)], axis=1)
    for g in range(m.shape[0]):
        y = oracle.eval(L[g:g + 1], m[g:g + 1], w[g:g + 1], x, tile=50)
        V3 = T[g].T @ T[g]
        d = xp - mu[g]
        e = np.exp(-0.5 * np.einsum("qi,ij,qj->q", d, np.linalg.inv(V3), d))
        np.testing.assert_allclose(y, wc[g][None, :] * e[:, None], rtol=1e-9, atol=1e-300)
        assert np.allclose(np.triu(T[g], 1), 0.0)
    # diagonal factor
    Ld = np.diag([0.3, 0.5, 0.2, 0.4, 0.25, 0.6])[None]
    md = np.array([[0.1, -0.2, 0.3, 0.0, 0.5, -0.4]])
    wd = np.array([[0.7, 0.2, 1.3]])
    mu, T, wc = oracle.condition(Ld, md, wd, xc)
    np.testing.assert_allclose(mu[0], md[0, :3], rtol=1e-14)
    np.testing.assert_allclose(T[0], np.diag(np.diag(Ld[0])[:3]), rtol=1e-14)
    f = np.exp(-0.5 * np.sum(((xc - md[0, 3:]) / np.diag(Ld[0])[3:]) ** 2))
    np.testing.assert_allclose(wc[0], wd[0] * f, rtol=1e-14)


def test_conditioned_cull_is_sound(oracle):
    """The contract on position for the Gaussians restricted to xc drops a
    (tile, Gaussian) pair only if the N-D Gaussian's largest weight times its
    factor stays below the cutoff at every query of the tile (queries carry
    xc in their last N - 3 inputs); the lists are much shorter than the
    contract's on all N inputs."""
    N, G, Q, tile, k = 6, 300, 2048, 64, 8
    mix = synth.mixture(N, G, seed=31)
    L, m, w = oracle.activate(raw_from(oracle, mix))
    r = np.random.default_rng(32)
    xc = r.uniform(-0.5, 0.5, size=N - 3)
    xp = synth.queries_box(3, Q, 33).astype(np.float64)
    x = np.concatenate([xp, np.repeat(xc[None, :], Q, axis=0)], axis=1)
    proj = synth.projections(N, k, 34)
    cutoff = 1.0 / 255.0
    offs, ids = oracle.cull_contract(L, m, w, x, tile, proj, cutoff, 3.0, 64, xc=xc)
    offs_n, _ = oracle.cull_contract(L, m, w, x, tile, proj, cutoff, 3.0, 64)
    assert offs[-1] < 0.5 * offs_n[-1]
    T = offs.size - 1
    keep = np.zeros((T, G), dtype=bool)
    for t in range(T):
        keep[t, ids[offs[t]:offs[t + 1]]] = True
    A = np.linalg.inv(L @ np.transpose(L, (0, 2, 1)))
    for g in range(G):
        d = x - m[g]
        s = np.einsum("qi,ij,qj->q", d, A[g], d).reshape(T, tile)
        contrib = w[g].max() * np.exp(-0.5 * s)
        assert np.all(contrib[~keep[:, g]] < cutoff), g


def test_conditioned_cull_interval_for_correlated_factors(oracle):
    """Conditioned cull with strongly correlated factors, one projection and
    one query per tile: along r (the projection's position components) a
    query stays a candidate exactly when its distance to r . mu is within
    3 sqrt(r^T V3 r), up to the contract's one bucket of slack on each side.
    mu and V3 come from the textbook precision-form conditional (numpy):
    V3 = A_pp^-1 and mu = m_p - A_pp^-1 A_pc (xc - m_c), A = (L L^T)^-1."""
    r = np.random.default_rng(41)
    N, G, Q, B = 4, 12, 4000, 256
    P = N * (N + 1) // 2
    th = np.zeros((G, P))
    for i in range(N):
        for j in range(i + 1):
            idx = i * (i + 1) // 2 + j
            th[:, idx] = np.log(r.uniform(0.05, 0.2, G)) if i == j else r.choice([-3.0, 3.0], G)
    mix = _raw_single_rows(N, r.uniform(-0.3, 0.3, (G, N)), th, np.ones(G), np.zeros((G, 3)))
    L, m, w = oracle.activate(raw_from(oracle, mix))
    xc = np.array([0.1])
    xp = r.uniform(-1.5, 1.5, size=(Q, 3))
    x = np.concatenate([xp, np.repeat(xc[None, :], Q, axis=0)], axis=1)
    n_in = n_out = 0
    for trial in range(4):
        proj = synth.projections(N, 1, 50 + trial)
        r3 = proj[0, :3].astype(np.float64)
        offs, ids = oracle.cull_contract(L, m, w, x, 1, proj, 0.0, 3.0, B, xc=xc)
        keep = np.zeros((Q, G), dtype=bool)
        for t in range(Q):
            keep[t, ids[offs[t]:offs[t + 1]]] = True
        v = xp @ r3
        h = (v.max() - v.min()) / B
        for g in range(G):
            A = np.linalg.inv(L[g] @ L[g].T)
            App, Apc = A[:3, :3], A[:3, 3:]
            mu = m[g, :3] - np.linalg.solve(App, Apc @ (xc - m[g, 3:]))
            half = 3.0 * math.sqrt(r3 @ np.linalg.solve(App, r3))
            dist = np.abs(v - r3 @ mu)
            inside = dist < half * (1 - 1e-5) - 1e-5
            outside = dist > half + 2.0 * h + 1e-4
            assert keep[inside, g].all(), (trial, g)
            assert not keep[outside, g].any(), (trial, g)
            n_in += int(inside.sum())
            n_out += int(outside.sum())
    assert n_in > 1000 and n_out > 1000


def _raw_single_rows(N, means, thetas, alphas, gammas):
    return {"mean": np.asarray(means, np.float64).reshape(-1, N),
            "theta": np.asarray(thetas, np.float64).reshape(len(alphas), -1),
            "alpha_raw": np.log(np.asarray(alphas, np.float64)),
            "color_raw": np.asarray(gammas, np.float64).reshape(-1, 3)}


def test_cull_exact_is_tight_in_one_dimension(oracle):
    """N = 1 with one query per tile: the projection test is exact, so the
    kept pairs are exactly those whose contribution w_max e^{-s/2} reaches
    the cutoff (the radius sqrt(2 ln(w_max / cutoff)) of the cutoff reading
    of Eq. 5)."""
    r = np.random.default_rng(12)
    G, Q, cutoff = 30, 400, 1.0 / 255.0
    sig = np.exp(r.uniform(np.log(0.02), np.log(0.3), size=G))
    mix = _raw_single_rows(1, r.uniform(-1, 1, G), np.log(sig), r.uniform(0.01, 1.0, G),
                           r.normal(size=(G, 3)))
    raw = raw_from(oracle, mix)
    L, m, w = oracle.activate(raw)
    x = np.linspace(-1.2, 1.2, Q).reshape(Q, 1)
    keep = oracle.cull_exact(L, m, w, x, 1, np.array([[1.0]]), cutoff, 3.0)
    contrib = w.max(axis=1)[None, :] * np.exp(-0.5 * ((x - m[:, 0][None, :]) / sig[None, :]) ** 2)
    clear = np.abs(contrib / cutoff - 1.0) > 1e-9
    assert np.array_equal(keep[clear].astype(bool), (contrib >= cutoff)[clear])
    assert 0 < keep.sum() < keep.size


def test_child_radius_floor_in_one_dimension(oracle):
    """Reading R7 of Section 3.3: a child (evaluated index >= n_parents)
    keeps a radius of at least child_k_min sigma, also when its largest
    weight is below the cutoff (it starts negligible and must still be
    optimised where it spans its parent); parents keep the cutoff radius.
    N = 1 with one query per tile makes the test exact: a dim child is kept
    exactly within child_k_min sigma of its mean, a bright child where its
    contribution reaches the cutoff or within child_k_min sigma, whichever
    is wider, a dim parent nowhere; without the floor a dim child is kept
    nowhere."""
    r = np.random.default_rng(13)
    G, Q, cutoff, kmin = 24, 500, 1.0 / 255.0, 3.0
    sig = np.exp(r.uniform(np.log(0.02), np.log(0.3), size=2 * G))
    # per group (parents, children): a third dim, a third just above the
    # cutoff (cutoff radius below kmin), a third bright (radius above kmin)
    wmax = np.concatenate([r.uniform(1e-4, 3e-3, G // 3), r.uniform(5e-3, 2e-2, G // 3),
                           r.uniform(0.3, 1.0, G - 2 * (G // 3))])
    wmax = np.concatenate([wmax, r.permutation(wmax)])
    w = wmax[:, None] * np.array([[1.0, 0.5, 0.25]])
    L = sig.reshape(-1, 1, 1)
    m = r.uniform(-1, 1, size=(2 * G, 1))
    x = np.linspace(-1.3, 1.3, Q).reshape(Q, 1)
    proj = np.array([[1.0]])
    keep = oracle.cull_exact(L, m, w, x, 1, proj, cutoff, 3.0, n_parents=G, child_k_min=kmin)
    plain = oracle.cull_exact(L, m, w, x, 1, proj, cutoff, 3.0)
    dist = np.abs(x - m[:, 0][None, :]) / sig[None, :]            # [Q, Ge] in sigmas
    kcut = np.where(wmax > cutoff, np.sqrt(2.0 * np.log(np.maximum(wmax, cutoff) / cutoff)), -1.0)
    radius = np.concatenate([kcut[:G], np.maximum(kcut[G:], kmin)])
    clear = np.abs(dist / np.maximum(radius, 1e-9)[None, :] - 1.0) > 1e-9
    want = dist <= radius[None, :]
    assert np.array_equal(keep[clear].astype(bool), want[clear])
    # parents: the floor changes nothing; dim children: kept only with it
    assert np.array_equal(keep[:, :G], plain[:, :G])
    dim_child = G + np.nonzero(wmax[G:] <= cutoff)[0]
    assert dim_child.size and keep[:, dim_child].any() and not plain[:, dim_child].any()
    # every dropped contribution stays below the cutoff
    contrib = wmax[None, :] * np.exp(-0.5 * dist ** 2)
    assert np.all(contrib[keep == 0] < cutoff)


def test_child_radius_floor_contract_is_conservative(oracle):
    """With children and the radius floor, the FP32 contract keeps every pair
    the exact test keeps (6-D, several projections), the dim children are
    evaluated, and every dropped pair's contribution is below the cutoff."""
    tile, cutoff = 64, 1.0 / 255.0
    mix, x, proj = _cull_case(seed=4, G=40)
    ch = synth.children(6, 40, 5, spread=0.05, brightness=(0.0009, 0.0011))
    L, m, w = oracle.activate(raw_from(oracle, mix, ch))
    G = 40
    keep = oracle.cull_exact(L, m, w, x, tile, proj, cutoff, 3.0, n_parents=G, child_k_min=3.0)
    offs, ids = oracle.cull_contract(L, m, w, x, tile, proj, cutoff, 3.0, 64, n_parents=G,
                                     child_k_min=3.0)
    T, Ge = keep.shape
    contract = np.zeros_like(keep)
    for t in range(T):
        contract[t, ids[offs[t]:offs[t + 1]]] = 1
    assert np.all(contract >= keep)
    assert keep[:, G:].any(), "children below the cutoff must be evaluated somewhere"
    for g in range(Ge):
        A = np.linalg.inv(L[g] @ L[g].T)
        d = x - m[g]
        s = np.einsum("qi,ij,qj->q", d, A, d).reshape(T, tile)
        contrib = w[g].max() * np.exp(-0.5 * s)
        assert np.all(contrib[contract[:, g] == 0] < cutoff)
        if g >= G:  # inside 3 sigma of a child: kept
            assert np.all(contract[:, g][(s <= 9.0).any(axis=1)] == 1)


def test_cull_sound_for_correlated_factors(oracle):
    """Strongly correlated factors (off-diagonals near +-1, small diagonals):
    the projected width must be |L^T r| (r^T V r), and one query per tile
    makes the test tight enough for a wrong width to drop kept pairs."""
    r = np.random.default_rng(13)
    for N in (2, 3):
        G, k = 12, 32
        P = N * (N + 1) // 2
        th = np.zeros((G, P))
        for i in range(N):
            for j in range(i + 1):
                idx = i * (i + 1) // 2 + j
                th[:, idx] = np.log(r.uniform(0.02, 0.08, G)) if i == j else r.choice([-3.5, 3.5], G)
        mix = _raw_single_rows(N, r.uniform(-0.5, 0.5, (G, N)), th, np.ones(G), np.zeros((G, 3)))
        raw = raw_from(oracle, mix)
        L, m, w = oracle.activate(raw)
        x = r.uniform(-1.5, 1.5, size=(3000, N))
        proj = synth.projections(N, k, 14 + N)
        keep = oracle.cull_exact(L, m, w, x, 1, proj, 0.0, 3.0)
        for g in range(G):
            A = np.linalg.inv(L[g] @ L[g].T)
            d = x - m[g]
            s = np.einsum("qi,ij,qj->q", d, A, d)
            assert np.all(s[keep[:, g] == 0] > 9.0)
            assert keep[s < 9.0, g].all()


def test_contract_bucket_slack(oracle):
    """The contract's one bucket of slack on each side of a Gaussian: with
    queries spanning [0, 1] in 10 buckets, a Gaussian covering [0.52, 0.58]
    (bucket 5) is a candidate of tiles in buckets 4..6 and of no other."""
    N = 1
    mix = _raw_single_rows(1, [0.55], [math.log(0.01)], [1.0], [[0.0, 0.0, 0.0]])
    raw = raw_from(oracle, mix)
    L, m, w = oracle.activate(raw)
    # ten tiles of two queries, tile b spanning [b/10 + 0.02, b/10 + 0.08];
    # the end points 0 and 1 pin the global range
    xs = [0.0, 0.01]
    for b in range(1, 9):
        xs += [b / 10 + 0.02, b / 10 + 0.08]
    xs += [0.99, 1.0]
    x = np.array(xs).reshape(-1, 1)
    offs, ids = oracle.cull_contract(L, m, w, x, 2, np.array([[1.0]]), 0.0, 3.0, 10)
    kept = [t for t in range(10) if offs[t + 1] > offs[t]]
    assert kept == [4, 5, 6]
    keep = oracle.cull_exact(L, m, w, x, 2, np.array([[1.0]]), 0.0, 3.0)
    assert np.nonzero(keep[:, 0])[0].tolist() == [5]


def test_cull_culled_sum_error_bound(oracle):
    """Culled sum vs dense sum: the difference equals the dropped terms, each
    below the cutoff (Eq. 5 with the cutoff radius)."""
    tile, cutoff = 64, 1.0 / 255.0
    mix, x, proj = _cull_case(seed=3)
    raw = raw_from(oracle, mix)
    L, m, w = oracle.activate(raw)
    offs, ids = oracle.cull_contract(L, m, w, x, tile, proj, cutoff, 3.0, 64)
    yd = oracle.eval(L, m, w, x, tile)
    yc = oracle.eval(L, m, w, x, tile, offs, ids)
    diff = yd - yc
    assert np.all(diff >= -1e-12)
    T = len(offs) - 1
    ndrop = np.array([L.shape[0] - (offs[t + 1] - offs[t]) for t in range(T)])
    bound = np.repeat(ndrop, tile)[:, None] * cutoff
    assert np.all(diff <= bound + 1e-12)


def test_cull_infinite_radius_keeps_everything(oracle):
    """k -> infinity: nothing is culled; lists are all ids in order."""
    tile = 128
    mix, x, proj = _cull_case(seed=4, G=40, Q=600)
    raw = raw_from(oracle, mix)
    L, m, w = oracle.activate(raw)
    offs, ids = oracle.cull_contract(L, m, w, x, tile, proj, 0.0, 1e30, 64)
    T = len(offs) - 1
    assert offs[-1] == T * 40
    for t in range(T):
        assert np.array_equal(ids[offs[t]:offs[t + 1]], np.arange(40))
    keep = oracle.cull_exact(L, m, w, x, tile, proj, 0.0, 1e30)
    assert keep.all()


def test_cull_no_projections_is_dense(oracle):
    """k = 0 projections: every live Gaussian is a candidate everywhere."""
    mix, x, proj = _cull_case(seed=5, G=30, Q=300)
    raw = raw_from(oracle, mix)
    L, m, w = oracle.activate(raw)
    offs, ids = oracle.cull_contract(L, m, w, x, 100, np.zeros((0, 6)), 0.0, 3.0, 64)
    assert offs[-1] == 3 * 30


# ---- loss and gradient ------------------------------------------------------

def test_loss_gradient_by_differences(oracle):
    """dl/dy from the loss by central differences (the loss is quadratic, so
    the difference is exact up to rounding)."""
    r = np.random.default_rng(0)
    y, t = r.normal(size=(7, 3)), r.normal(size=(7, 3))
    l0, gbar = oracle.loss_l2(y, t)
    assert abs(l0 - np.mean((y - t) ** 2)) < 1e-15
    for i in range(7):
        for c in range(3):
            yp, ym = y.copy(), y.copy()
            yp[i, c] += 1e-3
            ym[i, c] -= 1e-3
            fd = (oracle.loss_l2(yp, t)[0] - oracle.loss_l2(ym, t)[0]) / 2e-3
            assert abs(fd - gbar[i, c]) < 1e-10


def test_relative_l2_closed_form_and_gradient(oracle):
    """Relative L2 (Section 4.1, reading (y - t)^2 / (y^2 + eps) with the
    denominator held constant): a hand-computed two-output example, the
    eps -> 0 limit (squared relative error), invariance under scaling y, t by
    s with eps by s^2, and dl/dy by central differences of the loss with the
    denominator frozen at the unperturbed outputs."""
    # Q = 1: y = (1, 2, 0), t = (0, 1, 1), eps = 1:
    # (1/2 + 1/5 + 1/1) / 3 = 1.7 / 3;  gbar = 2 d / den / 3 = (1/3, 2/15, -2/3)
    y = np.array([[1.0, 2.0, 0.0]])
    t = np.array([[0.0, 1.0, 1.0]])
    l0, g0 = oracle.loss_rel_l2(y, t, eps=1.0)
    assert abs(l0 - 1.7 / 3.0) < 1e-15
    np.testing.assert_allclose(g0, [[1.0 / 3.0, 2.0 / 15.0, -2.0 / 3.0]], rtol=1e-14)
    r = np.random.default_rng(5)
    y = r.uniform(0.5, 2.0, size=(9, 3))
    t = r.uniform(0.0, 2.0, size=(9, 3))
    l1, _ = oracle.loss_rel_l2(y, t, eps=0.0)
    assert abs(l1 - np.mean(((y - t) / y) ** 2)) < 1e-14
    ls, _ = oracle.loss_rel_l2(7.0 * y, 7.0 * t, eps=49.0 * 1e-2)
    lr, gr = oracle.loss_rel_l2(y, t, eps=1e-2)
    assert abs(ls - lr) < 1e-14 * abs(lr) + 1e-16
    den = y ** 2 + 1e-2  # frozen denominator
    f = lambda yy: np.sum((yy - t) ** 2 / den) / y.size
    for i in range(9):
        for c in range(3):
            yp, ym = y.copy(), y.copy()
            yp[i, c] += 1e-3
            ym[i, c] -= 1e-3
            assert abs((f(yp) - f(ym)) / 2e-3 - gr[i, c]) < 1e-11


def _fd_check(oracle, raw, x, target, tile, offs, ids, n_samples, seed, h=1e-3, rtol=2e-5):
    y = oracle.eval(*oracle.activate(raw), x, tile, offs, ids)
    _, gbar = oracle.loss_l2(y, target)
    g = oracle.grad(raw, x, tile, offs, ids, gbar)
    r = np.random.default_rng(seed)
    names = ["mean", "theta", "alpha_raw", "color_raw", "u_theta", "m_u", "c_alpha_raw",
             "c_color_raw"]
    names = names if raw.has_children else names[:4]
    scale = max(np.abs(getattr(g, n)).max() for n in names)
    worst = 0.0
    for s in range(n_samples):
        n = names[s % len(names)]
        arr = getattr(raw, n)
        idx = tuple(r.integers(0, d) for d in arr.shape)
        old = arr[idx]

        def central(hh):
            arr[idx] = old + hh
            lp = oracle.loss_of_raw(raw, x, target, tile, offs, ids)
            arr[idx] = old - hh
            lm = oracle.loss_of_raw(raw, x, target, tile, offs, ids)
            arr[idx] = old
            return (lp - lm) / (2 * hh)

        # central differences at h and h/2 combined by Richardson
        # extrapolation: truncation O(h^4) instead of O(h^2)
        fd = (4.0 * central(h / 2) - central(h)) / 3.0
        an = getattr(g, n)[idx]
        err = abs(fd - an) / (abs(an) + 1e-3 * scale)
        worst = max(worst, err)
        assert err < rtol, (n, idx, fd, an)
    return worst


def test_gradient_central_differences_dense(oracle):
    """Analytic gradient = central differences (h = 1e-3) on raw parameters,
    parents and children, dense evaluation."""
    N, G, Q, tile = 4, 12, 300, 100
    mix = synth.mixture(N, G, seed=30)
    for key in mix:  # widen the Gaussians so every parameter matters
        mix[key] = mix[key].astype(np.float64)
    mix["theta"][:, [0, 2, 5, 9]] += 1.0
    ch = synth.children(N, G, seed=31)
    raw = raw_from(oracle, mix, ch)
    x = synth.queries_box(N, Q, 32).astype(np.float64)
    target = synth.targets_uniform(Q, 33)
    _fd_check(oracle, raw, x, target, tile, None, None, 64, seed=1)


def test_gradient_central_differences_culled(oracle):
    """Same, with candidate lists from the contract frozen (the culled loss
    is discontinuous at cull boundaries, so the lists must not move)."""
    N, G, Q, tile = 6, 40, 512, 64
    mix = synth.mixture(N, G, seed=40)
    ch = synth.children(N, G, seed=41, spread=0.2)
    raw = raw_from(oracle, mix, ch)
    L, m, w = oracle.activate(raw)
    x = synth.queries_box(N, Q, 42).astype(np.float64)
    proj = synth.projections(N, 8, 43)
    offs, ids = oracle.cull_contract(L, m, w, x, tile, proj, 1.0 / 255.0, 3.0, 64)
    assert 0 < offs[-1] < (Q // tile) * 2 * G
    target = synth.targets_uniform(Q, 44)
    _fd_check(oracle, raw, x, target, tile, offs, ids, 64, seed=2)


# ---- Adam and densification ---------------------------------------------------

def test_adam_first_step_closed_form(oracle):
    """From zero moments the bias-corrected first step is
    -lr g / (|g| + eps)."""
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    p, m1, m2 = oracle.adam(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, 0.01)
    np.testing.assert_allclose(p, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    # second step with the same gradient: m_hat = g, v_hat = g^2 again
    p2, _, _ = oracle.adam(p, g, m1, m2, 2, 0.01)
    np.testing.assert_allclose(p2 - p, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-9)


def _mixture_output(oracle, raw, x):
    L, m, w = oracle.activate(raw)
    return oracle.eval(L, m, w, x)


def test_densify_first_phase_adds_negligible_children(oracle):
    """Section 3.3: the first refinement gives every Gaussian a child with a
    negligible contribution spanning its parent; nothing materialises and
    the output moves by at most the children's weights."""
    N, G, cap = 6, 20, 30
    mix = synth.mixture(N, G, seed=50)
    raw = raw_from(oracle, mix)
    x = synth.queries_box(N, 200, 51).astype(np.float64)
    noise = synth.noise(cap, N, 52)
    t = 0.01
    new, Gn, flag = oracle.densify(raw, cap, math.log(t), math.log(t / 10), noise)
    assert Gn == G and not flag.any()
    after = oracle.Raw.from_arrays([a[:Gn] for a in new.arrays()], True)
    y0 = _mixture_output(oracle, raw, x)
    y1 = _mixture_output(oracle, after, x)
    wc = np.exp(after.c_alpha_raw)
    assert np.all(np.abs(y1 - y0) <= wc.sum() + 1e-12)
    assert np.all(wc < 2 * t / 10 * math.exp(0.5))  # negligible brightness


def test_densify_materialisation_preserves_mixture(oracle):
    """Section 3.3: a materialised child keeps exactly the Gaussian it was
    (L = L_p U, m = L_p m_u + m_p, own weights); only the fresh children add
    their negligible weights."""
    N, G, cap = 6, 25, 60
    mix = synth.mixture(N, G, seed=60)
    ch = synth.children(N, G, seed=61, spread=0.1, brightness=(0.001, 0.05))
    raw = raw_from(oracle, mix, ch)
    x = synth.queries_box(N, 300, 62).astype(np.float64)
    noise = synth.noise(cap, N, 63)
    t = 0.01
    a_thr = float(np.float32(math.log(t)))
    new, Gn, flag = oracle.densify(raw, cap, a_thr, math.log(t / 10), noise)
    nflag = int((raw.c_alpha_raw > a_thr).sum())
    assert 0 < nflag <= cap - G and Gn == G + nflag
    assert np.array_equal(flag.astype(bool), raw.c_alpha_raw > a_thr)
    after = oracle.Raw.from_arrays([a[:Gn] for a in new.arrays()], True)
    y0 = _mixture_output(oracle, raw, x)
    y1 = _mixture_output(oracle, after, x)
    fresh = np.concatenate([np.nonzero(flag)[0], np.arange(G, Gn)])
    wfresh = np.exp(after.c_alpha_raw[fresh]).sum()
    assert np.all(np.abs(y1 - y0) <= wfresh + 1e-9)
    # the materialised rows reproduce the old children exactly
    Lb, mb, wb = oracle.activate(raw)
    La, ma, wa = oracle.activate(after)
    for r_, g in enumerate(np.nonzero(flag)[0]):
        np.testing.assert_allclose(La[G + r_], Lb[G + g], rtol=1e-9, atol=1e-12)
        np.testing.assert_allclose(ma[G + r_], mb[G + g], rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(wa[G + r_], wb[G + g], rtol=1e-12)


def test_densify_capacity_keeps_brightest(oracle):
    """When more children qualify than rows remain, the brightest win."""
    N, G, cap = 3, 10, 13
    mix = synth.mixture(N, G, seed=70)
    ch = synth.children(N, G, seed=71)
    ch["c_alpha_raw"] = np.log(np.array([0.5, 0.02, 0.3, 0.001, 0.9, 0.05, 0.2, 0.002, 0.6, 0.04]))
    raw = raw_from(oracle, mix, ch)
    new, Gn, flag = oracle.densify(raw, cap, math.log(0.01), math.log(0.001), synth.noise(cap, N, 1))
    assert Gn == cap
    assert sorted(np.nonzero(flag)[0].tolist()) == [0, 4, 8]
