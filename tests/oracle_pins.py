"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each ``pin_*`` takes a loaded oracle (``oracle.OracleLib``) and raises
AssertionError when the oracle disagrees.  None of them re-types the oracle's
own formulas: they check closed forms, invariants, library routines of other
origin (numpy's FFT), brute force in the spatial domain and exhaustive scans.
``test_oracle_pins.py`` runs them on the committed oracle and
``test_oracle_mutants.py`` checks that planted mistakes make at least one fail.
"""
from __future__ import annotations

import os

import numpy as np

S = 32
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rand_block(seed, S=S, p_known=0.5):
    rng = np.random.default_rng(seed)
    f = rng.uniform(0, 255, (S, S))
    known = rng.random((S, S)) < p_known
    known[S // 2, S // 2] = True
    return f, known


def _neg(S):
    return (-np.arange(S)) % S


def _model_history(res, gamma, K, S=S):
    """G^(nu) for nu = 0..K from the selected indices and coefficients."""
    G = np.zeros((K + 1, S, S), complex)
    for nu in range(K):
        G[nu + 1] = G[nu]
        idx = res["seq"][nu]
        if idx >= 0:
            G[nu + 1].flat[idx] += gamma * res["p"][nu] * S * S
    return G


def _conj_model_history(res, gamma, K, S=S):
    """G^(nu) of the conjugate-pair ablation: a = gamma p at the selected index
    and conj(a) at its conjugate index (once for a self-conjugate index)."""
    G = np.zeros((K + 1, S, S), complex)
    n = _neg(S)
    for nu in range(K):
        G[nu + 1] = G[nu]
        idx = int(res["seq"][nu])
        if idx < 0:
            continue
        u, v = divmod(idx, S)
        a = gamma * res["p"][nu] * S * S
        G[nu + 1][u, v] += a
        if (n[u], n[v]) != (u, v):
            G[nu + 1][n[u], n[v]] += np.conj(a)
    return G


def _energy(fw_tilde, w, G):
    """Weighted residual energy of Eqs. (3)-(4) in the spatial domain for a
    model spectrum G (g = complex inverse DFT by numpy)."""
    g = np.fft.ifft2(G)
    r = fw_tilde - g
    return float(np.sum(np.abs(r) ** 2 * w))


# --- Eq. (5), Eq. (9): closed-form values --------------------------------

def load_closed_forms():
    """Closed-form values written out by hand in tests/golden/closed_forms.txt."""
    rows = []
    with open(os.path.join(GOLDEN, "closed_forms.txt")) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            kind, S_, rho, a, b, value = line.split()
            rows.append((kind, int(S_), float(rho), int(a), int(b), eval(value, {"sqrt": np.sqrt})))
    return rows


def pin_weights_closed_form(lib):
    rows = load_closed_forms()
    assert rows
    for kind, S_, rho, a, b, value in rows:
        if kind == "w":
            got = lib.spatial_weight(S_, rho)[a, b]
        elif kind == "wf":
            got = lib.freq_weight(S_)[a, b]
        else:
            raise AssertionError(kind)
        assert abs(got - value) <= 1e-13 * max(1.0, abs(value)), (kind, S_, a, b, got, value)


def pin_weight_symmetries(lib):
    for S_ in (8, 16, 24, 32):
        w = lib.spatial_weight(S_, 0.7)
        # symmetric about the support centre in both axes and under transposition
        assert np.array_equal(w, w[::-1, :]) and np.array_equal(w, w[:, ::-1])
        assert np.array_equal(w, w.T)
        assert np.allclose(lib.spatial_weight(S_, 1.0), 1.0)
        wf = lib.freq_weight(S_)
        n = _neg(S_)
        assert np.allclose(wf, wf[n][:, n]) and np.allclose(wf, wf.T)
        # strictly largest at DC, zero at the highest frequency (S/2, S/2)
        assert wf[0, 0] == 1.0 and np.sum(wf >= 1.0) == 1
        assert abs(wf[S_ // 2, S_ // 2]) < 1e-15


# --- the 2-D DFT -------------------------------------------------------------

def pin_dft_against_numpy(lib):
    rng = np.random.default_rng(5)
    for S_ in (8, 16, 24, 32):
        x = rng.standard_normal((S_, S_)) * 50 + 10
        X = lib.dft2_real(x)
        ref = np.fft.fft2(x)
        assert np.max(np.abs(X - ref)) <= 1e-10 * np.max(np.abs(ref))
    # orientation: a single pixel at (m0, n0) has X[k, l] = e^{-j2pi(k m0 + l n0)/S}
    x = np.zeros((S, S)); x[3, 11] = 1.0
    k, l = np.mgrid[0:S, 0:S]
    assert np.allclose(lib.dft2_real(x), np.exp(-2j * np.pi * (k * 3 + l * 11) / S), atol=1e-13)


def pin_hermitian_exact(lib):
    f, known = _rand_block(11)
    res = lib.fsr_block(f, known, K=1)
    n = _neg(S)
    for X in (res["R0"], res["W"]):
        Xc = np.conj(X[n][:, n])
        assert np.array_equal(X.real, Xc.real) and np.array_equal(X.imag, Xc.imag)
    # conjugate pair tie at nu = 0: the lower linear index is selected
    idx = int(res["seq"][0]); u, v = divmod(idx, S)
    assert idx <= ((-u) % S) * S + (-v) % S


# --- Eq. (7) and the weighting spectrum -------------------------------------

def pin_initial_spectra(lib):
    f, known = _rand_block(12)
    res = lib.fsr_block(f, known, K=0)
    w = res["w"]
    w0 = lib.spatial_weight(S, 0.7)
    assert np.array_equal(w, np.where(known, w0, 0.0))
    assert np.allclose(res["R0"], np.fft.fft2(np.where(known, f, 0.0) * w), rtol=0, atol=1e-9)
    assert np.allclose(res["W"], np.fft.fft2(w), rtol=0, atol=1e-12)
    assert abs(res["W"][0, 0].real - w.sum()) < 1e-12


# --- Eqs. (3)-(12): brute force in the spatial domain -----------------------

def pin_residual_is_spatial_residual(lib):
    """R^(nu) = F2{(f~ - g^(nu)) w}, g^(nu) = IDFT2(G^(nu)) (Eqs. 4, 6)."""
    for seed, gamma, fw in ((13, 0.5, True), (14, 0.3, False), (15, 1.0, True)):
        f, known = _rand_block(seed)
        K = 25
        res = lib.fsr_block(f, known, K=K, gamma=gamma, freq_weight=fw, history=True)
        G = _model_history(res, gamma, K)
        fw_tilde = np.where(known, f, 0.0)
        w = res["w"]
        scale = np.max(np.abs(res["R0"]))
        for nu in range(K + 1):
            g = np.fft.ifft2(G[nu])
            Rb = np.fft.fft2((fw_tilde - g) * w)
            assert np.max(np.abs(res["R_hist"][nu] - Rb)) <= 1e-10 * scale, (seed, nu)
        assert np.allclose(res["G"], G[K], rtol=0, atol=1e-9 * np.max(np.abs(G[K])))
        assert np.allclose(res["g"], np.fft.ifft2(G[K]), rtol=0, atol=1e-9 * np.max(np.abs(f)))


def pin_argmax_exhaustive(lib):
    """Eq. (8): each selected index is the first maximum of the full scan."""
    wf = lib.freq_weight(S)
    for seed, fw in ((16, True), (17, False)):
        f, known = _rand_block(seed)
        K = 30
        res = lib.fsr_block(f, known, K=K, freq_weight=fw, history=True)
        for nu in range(K):
            obj = (wf if fw else 1.0) * np.abs(res["R_hist"][nu]) ** 2
            assert int(res["seq"][nu]) == int(np.argmax(obj)), (seed, nu)
            # the diagnostic gap to the best component that is not the pick's conjugate
            u, v = divmod(int(res["seq"][nu]), S)
            rest = obj.copy()
            rest[u, v] = rest[(-u) % S, (-v) % S] = -1.0
            gap = (obj[u, v] - rest.max()) / obj[u, v]
            assert abs(res["margin_nc"][nu] - gap) <= 1e-9, (seed, nu)


def pin_energy_decrease(lib):
    """Each step lowers E_w by exactly (2 gamma - gamma^2)|R(u,v)|^2 / W(0,0):
    the value that makes p of Eq. (10) the weighted projection onto phi_uv."""
    for seed, gamma in ((18, 0.5), (19, 0.8)):
        f, known = _rand_block(seed)
        K = 20
        res = lib.fsr_block(f, known, K=K, gamma=gamma, history=True)
        G = _model_history(res, gamma, K)
        fw_tilde = np.where(known, f, 0.0)
        w = res["w"]
        W0 = w.sum()
        E = [_energy(fw_tilde, w, G[nu]) for nu in range(K + 1)]
        for nu in range(K):
            R = res["R_hist"][nu].flat[res["seq"][nu]]
            want = (2 * gamma - gamma ** 2) * abs(R) ** 2 / W0
            assert abs((E[nu] - E[nu + 1]) - want) <= 1e-9 * E[0], (seed, nu)


def pin_projection_optimal(lib):
    """With gamma = 1, perturbing the chosen coefficient only raises E_w (Eq. 3)."""
    f, known = _rand_block(20)
    res = lib.fsr_block(f, known, K=1, gamma=1.0)
    fw_tilde = np.where(known, f, 0.0)
    w = res["w"]
    E1 = _energy(fw_tilde, w, res["G"])
    idx = int(res["seq"][0])
    for d in (1e-3, -1e-3, 1e-3j, -1e-3j):
        G = res["G"].copy()
        G.flat[idx] += d * S * S
        assert _energy(fw_tilde, w, G) > E1


def pin_selected_component_shrinks(lib):
    f, known = _rand_block(21)
    gamma = 0.5
    res = lib.fsr_block(f, known, K=10, gamma=gamma, history=True)
    for nu in range(10):
        idx = res["seq"][nu]
        a = res["R_hist"][nu].flat[idx]; b = res["R_hist"][nu + 1].flat[idx]
        assert abs(b - (1 - gamma) * a) <= 1e-11 * abs(a)


# --- closed-form reconstructions ---------------------------------------------

def pin_dc_closed_form(lib):
    """Constant block c: DC every iteration and g = c (1 - (1 - gamma)^K)."""
    rng = np.random.default_rng(22)
    for c, gamma, K in ((7.0, 0.5, 3), (200.0, 0.3, 40), (31.5, 0.9, 12)):
        known = rng.random((S, S)) < 0.3
        known[0, 0] = True
        res = lib.fsr_block(np.full((S, S), c), known, K=K, gamma=gamma)
        assert np.all(res["seq"] == 0)
        want = c * (1 - (1 - gamma) ** K)
        assert np.max(np.abs(res["g"] - want)) <= 1e-11 * c


def pin_single_basis_recovery(lib):
    """rho = 1, all pixels known, gamma = 1, no frequency weighting: a real
    cosine (a conjugate pair of basis images) is recovered exactly in two
    iterations, lower index of the pair first."""
    m, n = np.mgrid[0:S, 0:S]
    for (u, v, A, ph) in ((3, 5, 40.0, 0.3), (1, 30, 12.5, -1.1), (7, 0, 3.0, 0.0)):
        f = A * np.cos(2 * np.pi * (u * m + v * n) / S + ph)
        res = lib.fsr_block(f, np.ones((S, S), bool), K=2, rho=1.0, gamma=1.0,
                            freq_weight=False)
        pair = sorted([u * S + v, ((-u) % S) * S + (-v) % S])
        assert list(res["seq"]) == pair, res["seq"]
        assert np.max(np.abs(res["g"] - f)) <= 1e-10 * A


# --- image level: tiling, write-back, edge cases -------------------------------

def _support(img, mask, b, B, L):
    H, Wd = img.shape
    nbx = -(-Wd // B)
    by, bx = divmod(b, nbx)
    S_ = B + 2 * L
    f = np.zeros((S_, S_)); kn = np.zeros((S_, S_), bool)
    for mm in range(S_):
        for nn in range(S_):
            y, x = by * B - L + mm, bx * B - L + nn
            if 0 <= y < H and 0 <= x < Wd and mask[y, x]:
                kn[mm, nn] = True
                f[mm, nn] = img[y, x]
    return f, kn, by, bx


def pin_tiling_matches_block_routine(lib):
    rng = np.random.default_rng(23)
    H, Wd, B, L, K = 37, 53, 4, 14, 15
    img = rng.uniform(0, 255, (H, Wd)).astype(np.float32)
    mask = (rng.random((H, Wd)) < 0.4).astype(np.uint8)
    nbx, nby = -(-Wd // B), -(-H // B)
    ids = np.array([0, 5, nbx - 1, nbx * 3 + 7, nbx * nby - 1, nbx * (nby - 1)])
    res = lib.fsr_image_blocks(img, mask, B=B, L=L, K=K, block_ids=ids, threads=1)
    for s, b in enumerate(ids):
        f, kn, by, bx = _support(img, mask, int(b), B, L)
        r = lib.fsr_block(f, kn, K=K)
        for a in range(B):
            for c in range(B):
                y, x = by * B + a, bx * B + c
                got = res["target"][s, a, c]
                if y >= H or x >= Wd:
                    assert np.isnan(got)
                elif mask[y, x]:
                    assert got == img[y, x]
                else:
                    assert abs(got - r["g"][L + a, L + c].real) <= 1e-9 * 255
        assert np.array_equal(res["seq"][s], r["seq"])


def pin_image_edge_cases(lib):
    from oracle import assemble_image  # placement helper only
    rng = np.random.default_rng(24)
    H, Wd = 21, 18
    img = rng.uniform(0, 255, (H, Wd)).astype(np.float32)
    mask = (rng.random((H, Wd)) < 0.5).astype(np.uint8)
    # known pixels are copied bit for bit; NaN at missing pixels is never read
    bad = img.copy(); bad[mask == 0] = np.nan
    r = lib.fsr_image_blocks(bad, mask, K=10, threads=2)
    out = assemble_image(r["target"], H, Wd, 4)
    assert np.all(np.isfinite(out))
    assert np.array_equal(out[mask == 1], img[mask == 1].astype(np.float64))
    # a fully known image comes back unchanged
    r = lib.fsr_image_blocks(img, np.ones_like(mask), K=10)
    assert np.array_equal(assemble_image(r["target"], H, Wd, 4), img.astype(np.float64))
    # K = 0: unknown pixels are 0
    r = lib.fsr_image_blocks(img, mask, K=0)
    out = assemble_image(r["target"], H, Wd, 4)
    assert np.all(out[mask == 0] == 0.0)
    # no known pixel anywhere: every block is skipped, output 0
    r = lib.fsr_image_blocks(img, np.zeros_like(mask), K=5)
    assert r["n_empty"] == 6 * 5 and np.all(r["seq"] == -1)
    assert np.all(assemble_image(r["target"], H, Wd, 4) == 0.0)


def pin_block_ignores_unknown_values(lib):
    """Eq. (2): values at unknown pixels never enter the result."""
    f, known = _rand_block(25)
    a = lib.fsr_block(f, known, K=12)
    f2 = f.copy(); f2[~known] = np.nan
    b = lib.fsr_block(f2, known, K=12)
    assert np.array_equal(a["seq"], b["seq"]) and np.array_equal(a["g"], b["g"])


def pin_small_supports(lib):
    """The same facts at the support sizes of the support-size study (S = 4,
    8, 16, 24): spatial-domain residual, exhaustive argmax, exact energy
    decrease, exact recovery of a cosine and the tiling of an image with
    L = (S - 4) / 2."""
    for S_ in (4, 8, 16, 24):
        wf = lib.freq_weight(S_)
        # exactly Hermitian spectra at every support size (the ties of nu = 0 are exact)
        r0 = lib.fsr_block(*_rand_block(60 + S_, S=S_), K=1)
        n_ = _neg(S_)
        for X in (r0["R0"], r0["W"]):
            assert np.array_equal(X, np.conj(X[n_][:, n_])), S_
        for seed, gamma in ((40 + S_, 0.5), (41 + S_, 0.8)):
            f, known = _rand_block(seed, S=S_)
            K = 12
            res = lib.fsr_block(f, known, K=K, gamma=gamma, history=True)
            G = _model_history(res, gamma, K, S=S_)
            fw_tilde = np.where(known, f, 0.0)
            w = res["w"]
            W0 = w.sum()
            scale = np.max(np.abs(res["R0"]))
            E = [_energy(fw_tilde, w, G[nu]) for nu in range(K + 1)]
            for nu in range(K):
                Rb = np.fft.fft2((fw_tilde - np.fft.ifft2(G[nu])) * w)
                assert np.max(np.abs(res["R_hist"][nu] - Rb)) <= 1e-10 * scale, (S_, seed, nu)
                obj = wf * np.abs(res["R_hist"][nu]) ** 2
                assert int(res["seq"][nu]) == int(np.argmax(obj)), (S_, seed, nu)
                R = res["R_hist"][nu].flat[res["seq"][nu]]
                want = (2 * gamma - gamma ** 2) * abs(R) ** 2 / W0
                assert abs((E[nu] - E[nu + 1]) - want) <= 1e-9 * E[0], (S_, seed, nu)
        m, n = np.mgrid[0:S_, 0:S_]
        u, v = 1, S_ // 2 - 1
        f = 20.0 * np.cos(2 * np.pi * (u * m + v * n) / S_ + 0.4)
        res = lib.fsr_block(f, np.ones((S_, S_), bool), K=2, rho=1.0, gamma=1.0, freq_weight=False)
        assert list(res["seq"]) == sorted([u * S_ + v, ((-u) % S_) * S_ + (-v) % S_])
        assert np.max(np.abs(res["g"] - f)) <= 1e-10 * 20.0
        # image tiling with B = 4, L = (S - 4) / 2
        rng = np.random.default_rng(50 + S_)
        H, Wd, B, L, K = 23, 29, 4, (S_ - 4) // 2, 8
        img = rng.uniform(0, 255, (H, Wd)).astype(np.float32)
        mask = (rng.random((H, Wd)) < 0.4).astype(np.uint8)
        nbx, nby = -(-Wd // B), -(-H // B)
        ids = np.array([0, nbx - 1, nbx * 2 + 3, nbx * nby - 1])
        r = lib.fsr_image_blocks(img, mask, B=B, L=L, K=K, block_ids=ids, threads=1)
        for s_, b in enumerate(ids):
            f, kn, by, bx = _support(img, mask, int(b), B, L)
            rb = lib.fsr_block(f, kn, K=K)
            assert np.array_equal(r["seq"][s_], rb["seq"])
            for a_ in range(B):
                for c_ in range(B):
                    y, x = by * B + a_, bx * B + c_
                    if y < H and x < Wd and not mask[y, x]:
                        assert abs(r["target"][s_, a_, c_] - rb["g"][L + a_, L + c_].real) <= 1e-9 * 255


def pin_conj_pairs(lib):
    """The conjugate-pair ablation (the original FSR's real model; not the
    paper's Eqs. 11-12): the residual stays exactly Hermitian, equals the
    spatial-domain residual of the real model, the selection is the first
    maximum of the full scan, and each step lowers E_w by the closed form of
    a real pair update with a = gamma R/W0:
    2(2g - g^2)|R|^2/W0 - 2 g^2 Re(conj(R)^2 W[2u,2v])/W0^2, or
    (2g - g^2) R^2/W0 for a self-conjugate (u,v)."""
    for seed, gamma, S_ in ((70, 0.5, S), (71, 0.8, S), (72, 0.5, 16), (73, 0.5, 24)):
        f, known = _rand_block(seed, S=S_)
        K = 14
        res = lib.fsr_block(f, known, K=K, gamma=gamma, history=True, conj_pairs=True)
        n = _neg(S_)
        wf = lib.freq_weight(S_)
        fw_tilde = np.where(known, f, 0.0)
        w = res["w"]
        W0 = w.sum()
        Wsp = res["W"]
        G = _conj_model_history(res, gamma, K, S=S_)
        scale = np.max(np.abs(res["R0"]))
        E = [_energy(fw_tilde, w, G[nu]) for nu in range(K + 1)]
        selfconj = 0
        for nu in range(K):
            R = res["R_hist"][nu]
            assert np.array_equal(R, np.conj(R[n][:, n])), (S_, seed, nu)
            Rb = np.fft.fft2((fw_tilde - np.fft.ifft2(G[nu]).real) * w)
            assert np.max(np.abs(R - Rb)) <= 1e-10 * scale, (S_, seed, nu)
            obj = wf * np.abs(R) ** 2
            idx = int(res["seq"][nu])
            assert idx == int(np.argmax(obj)), (S_, seed, nu)
            u, v = divmod(idx, S_)
            Ru = R.flat[idx]
            if (n[u], n[v]) == (u, v):
                selfconj += 1
                want = (2 * gamma - gamma ** 2) * abs(Ru) ** 2 / W0
            else:
                want = (2 * (2 * gamma - gamma ** 2) * abs(Ru) ** 2 / W0
                        - 2 * gamma ** 2 * (np.conj(Ru) ** 2 * Wsp[(2 * u) % S_, (2 * v) % S_]).real / W0 ** 2)
            assert abs((E[nu] - E[nu + 1]) - want) <= 1e-9 * E[0], (S_, seed, nu)
        assert selfconj > 0 and selfconj < K   # both kinds of update were exercised
        assert np.max(np.abs(res["G"] - G[K])) <= 1e-9 * np.max(np.abs(G[K]))
        assert np.max(np.abs(res["g"] - np.fft.ifft2(G[K]))) <= 1e-9 * 255
        assert np.max(np.abs(res["g"].imag)) <= 1e-9 * 255
    # a real cosine, every pixel known, rho = gamma = 1: one pair recovers it
    m, n_ = np.mgrid[0:S, 0:S]
    u, v = 3, 5
    f = 20.0 * np.cos(2 * np.pi * (u * m + v * n_) / S + 0.4)
    res = lib.fsr_block(f, np.ones((S, S), bool), K=1, rho=1.0, gamma=1.0, freq_weight=False, conj_pairs=True)
    assert list(res["seq"]) == [min(u * S + v, ((-u) % S) * S + (-v) % S)]
    assert np.max(np.abs(res["g"] - f)) <= 1e-10 * 20.0


def pin_scaled_weights(lib):
    """The weight-scaled block routine (re-use form): w = scale * w0 of Eq.
    (5) with the scale per pixel, R0 = F2{f w} and W = F2{w} against numpy's
    FFT; scale 1 on the known set is the paper's block routine bit for bit;
    the energy identity of Eq. (10) holds with the scaled weights."""
    rng = np.random.default_rng(31)
    f = rng.uniform(0, 255, (S, S))
    scale = rng.choice([0.0, 0.25, 0.5, 1.0], (S, S))
    scale[S // 2, S // 2] = 1.0
    w0 = lib.spatial_weight(S, 0.7)
    res = lib.fsr_block(f, None, K=8, scale=scale, history=True)
    w = scale * w0
    assert np.allclose(res["w"], w, rtol=0, atol=1e-15)
    assert np.allclose(res["R0"], np.fft.fft2(f * w), rtol=0, atol=1e-9 * np.abs(np.fft.fft2(f * w)).max())
    assert np.allclose(res["W"], np.fft.fft2(w), rtol=0, atol=1e-12 * np.abs(np.fft.fft2(w)).max())
    # the residual is the spectrum of the weighted spatial residual (Eqs. 4, 6)
    G = _model_history(res, 0.5, 8)
    for nu in (0, 3, 8):
        g = np.fft.ifft2(G[nu])
        ref = np.fft.fft2((f - g) * w)
        assert np.allclose(res["R_hist"][nu], ref, rtol=0, atol=1e-9 * np.abs(ref).max())
    known = rng.random((S, S)) < 0.5
    a = lib.fsr_block(f, known, K=10)
    b = lib.fsr_block(f, None, K=10, scale=known.astype(np.float64))
    assert np.array_equal(a["seq"], b["seq"]) and np.array_equal(a["g"], b["g"])


def _reuse_support(img, mask, out, b, B, L, delta):
    """Support of block b in the re-use form, built from the definition:
    known pixels with scale 1, unknown pixels of earlier blocks in raster
    order with their final reconstruction and scale delta, the rest 0."""
    H, Wd = img.shape
    nbx = -(-Wd // B)
    by, bx = divmod(b, nbx)
    S_ = B + 2 * L
    f = np.zeros((S_, S_)); sc = np.zeros((S_, S_))
    for mm in range(S_):
        for nn in range(S_):
            y, x = by * B - L + mm, bx * B - L + nn
            if not (0 <= y < H and 0 <= x < Wd):
                continue
            if mask[y, x]:
                f[mm, nn], sc[mm, nn] = img[y, x], 1.0
            elif (y // B) * nbx + (x // B) < b:
                f[mm, nn], sc[mm, nn] = out[y, x], delta
    return f, sc, by, bx


def pin_reuse_form(lib):
    """Re-use of reconstructed pixels (the sequential form Sec. II leaves out;
    reading in fsr_oracle.c): with delta = 0 it is the independent-block
    oracle bit for bit; with delta > 0 every block equals the block routine
    run on its support built from the definition (raster order, earlier
    blocks' reconstructions at weight delta), on a non-square ragged image
    whose later blocks see earlier reconstructions in their supports."""
    from oracle import assemble_image  # placement helper only
    rng = np.random.default_rng(32)
    H, Wd, B, L, K = 29, 43, 4, 14, 12
    img = rng.uniform(0, 255, (H, Wd)).astype(np.float32)
    mask = (rng.random((H, Wd)) < 0.35).astype(np.uint8)
    ind = assemble_image(lib.fsr_image_blocks(img, mask, B=B, L=L, K=K, threads=1)["target"], H, Wd, B)
    r0 = lib.fsr_image_reuse(img, mask, B=B, L=L, K=K, delta=0.0)
    assert np.array_equal(r0["out"], ind)
    delta = 0.5
    r = lib.fsr_image_reuse(img, mask, B=B, L=L, K=K, delta=delta)
    out = r["out"]
    assert np.all(np.isfinite(out)) and np.array_equal(out[mask == 1], img[mask == 1].astype(np.float64))
    assert not np.array_equal(out, ind)           # re-used pixels change the result
    nbx, nby = -(-Wd // B), -(-H // B)
    for b in range(nbx * nby):
        f, sc, by, bx = _reuse_support(img, mask, out, b, B, L, delta)
        res = lib.fsr_block(f, None, K=K, scale=sc)
        assert np.array_equal(r["seq"][b], res["seq"]), b
        for a in range(B):
            for c in range(B):
                y, x = by * B + a, bx * B + c
                if y < H and x < Wd and not mask[y, x]:
                    assert abs(out[y, x] - res["g"][L + a, L + c].real) <= 1e-9 * 255, (b, a, c)
    # with the sequential result given as the source of re-used values, every
    # block sees the same support: the parallel evaluation is bit-identical
    par = lib.fsr_image_reuse(img, mask, B=B, L=L, K=K, delta=delta, given=out, threads=3)
    assert np.array_equal(par["out"], out) and np.array_equal(par["seq"], r["seq"])
    # a prefix of the raster order is computed alone, NaN beyond it
    part = lib.fsr_image_reuse(img, mask, B=B, L=L, K=K, delta=delta, nblocks=nbx * 3 + 2)
    done = np.zeros((H, Wd), bool)
    for b in range(nbx * 3 + 2):
        by, bx = divmod(b, nbx)
        done[by * B:by * B + B, bx * B:bx * B + B] = True
    done |= mask == 1
    assert np.array_equal(part["out"][done], out[done]) and np.all(np.isnan(part["out"][~done]))


ALL_PINS = [
    pin_weights_closed_form,
    pin_weight_symmetries,
    pin_dft_against_numpy,
    pin_hermitian_exact,
    pin_initial_spectra,
    pin_residual_is_spatial_residual,
    pin_argmax_exhaustive,
    pin_energy_decrease,
    pin_projection_optimal,
    pin_selected_component_shrinks,
    pin_dc_closed_form,
    pin_single_basis_recovery,
    pin_tiling_matches_block_routine,
    pin_image_edge_cases,
    pin_block_ignores_unknown_values,
    pin_small_supports,
    pin_conj_pairs,
    pin_scaled_weights,
    pin_reuse_form,
]
