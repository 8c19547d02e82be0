"""Pins for the FP64 oracle: checks against what the paper and the mathematics
fix, independent of the oracle's own code.

Every pin takes the oracle as a namespace ``O`` so that the mutation tests can
hand in a copy with one planted mistake and assert that some pin fails.
"""

from __future__ import annotations

import os

import numpy as np

from paper_2504_03373_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _lines(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def _crand(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _herm_pd(rng, B, M, cond=10.0):
    Q = synth.haar_unitary(rng, B, M)
    s = np.logspace(0, -np.log10(cond), M)
    return np.matmul(Q * s[None, None, :], np.conj(np.swapaxes(Q, 1, 2)))


# --------------------------------------------------------------------------
# correlation (eq. 2-3)
# --------------------------------------------------------------------------

def pin_correlation_golden(O):
    rows = _lines("correlation_2ch_hand.txt")
    X = np.zeros((2, 1, 2), complex)
    Rexp = np.zeros((1, 2, 2), complex)
    for r in rows:
        if r[0] == "X":
            X[int(r[1]), 0, int(r[2])] = float(r[3]) + 1j * float(r[4])
        else:
            Rexp[0, int(r[1]), int(r[2])] = float(r[3]) + 1j * float(r[4])
    assert np.allclose(O.correlation(X), Rexp, atol=1e-15)


def pin_correlation_bruteforce(O):
    rng = np.random.default_rng(11)
    T, B, M = 5, 3, 4
    X = _crand(rng, T, B, M)
    R = O.correlation(X)
    for b in range(B):
        for i in range(M):
            for j in range(M):
                acc = 0j
                for f in range(T):
                    acc += X[f, b, i] * X[f, b, j].conjugate()
                assert abs(R[b, i, j] - acc / T) < 1e-13


def pin_correlation_structure(O):
    rng = np.random.default_rng(12)
    X = _crand(rng, 7, 4, 6)
    R = O.correlation(X)
    assert np.allclose(R, np.conj(np.swapaxes(R, 1, 2)), atol=1e-14)
    w = np.linalg.eigvalsh(R)
    assert np.all(w >= -1e-12 * np.abs(w).max())
    # Rank is at most T when M > T.
    Xs = _crand(rng, 3, 2, 6)
    ws = np.linalg.eigvalsh(O.correlation(Xs))
    assert np.all(np.abs(ws[:, :3]) < 1e-12 * ws.max())
    # Frames combine by a T-weighted average (eq. 3's 1/T).
    X1, X2 = X[:3], X[3:]
    R12 = (3 * O.correlation(X1) + 4 * O.correlation(X2)) / 7
    assert np.allclose(R12, R, atol=1e-13)


# --------------------------------------------------------------------------
# whitening (eq. 4 left-hand side, Sec. III-B)
# --------------------------------------------------------------------------

def pin_whiten_golden(O):
    rows = _lines("whiten_2x2_hand.txt")
    mats = {"K": np.zeros((1, 2, 2), complex), "R": np.zeros((1, 2, 2), complex),
            "A": np.zeros((1, 2, 2), complex)}
    for r in rows:
        mats[r[0]][0, int(r[1]), int(r[2])] = float(r[3]) + 1j * float(r[4])
    assert np.allclose(O.whiten(mats["K"], mats["R"]), mats["A"], atol=1e-14)


def pin_whiten_solves(O):
    rng = np.random.default_rng(13)
    B, M = 5, 7
    K = _herm_pd(rng, B, M, cond=1e3)
    R = O.correlation(_crand(rng, 20, B, M))
    A = O.whiten(K, R)
    assert np.linalg.norm(np.matmul(K, A) - R) <= 1e-11 * np.linalg.norm(R)
    I = np.broadcast_to(np.eye(M), K.shape).astype(complex)
    assert np.allclose(O.whiten(I, R), R, atol=1e-14)
    Ach = np.matmul(O.inverse_by_cholesky(K), R)
    assert np.linalg.norm(Ach - A) <= 1e-9 * np.linalg.norm(A)


# --------------------------------------------------------------------------
# decomposition (eq. 4)
# --------------------------------------------------------------------------

def _faddeev_leverrier(C):
    """Characteristic polynomial coefficients of a small matrix by the
    Faddeev-LeVerrier recursion (traces and products only)."""
    n = C.shape[0]
    coeffs = [1.0 + 0j]
    Mk = np.zeros_like(C)
    I = np.eye(n)
    for k in range(1, n + 1):
        Mk = C @ Mk + coeffs[-1] * I
        ck = -np.trace(C @ Mk) / k
        coeffs.append(ck)
    return np.array(coeffs)


def pin_gsvd_golden(O):
    rows = _lines("svd_2x2_textbook.txt")
    A = np.zeros((1, 2, 2), complex)
    S = np.zeros(2)
    for r in rows:
        if r[0] == "A":
            A[0, int(r[1]), int(r[2])] = float(r[3]) + 1j * float(r[4])
        else:
            S[int(r[1])] = float(r[2])
    I = np.eye(2)[None].astype(complex)
    _, _, lam, _ = O.gsvd(I, A)
    assert np.allclose(lam[0], S, atol=1e-13)


def pin_gsvd_factorisation(O):
    rng = np.random.default_rng(14)
    B, M = 6, 8
    K = _herm_pd(rng, B, M, cond=1e2)
    R = O.correlation(_crand(rng, 30, B, M))
    A, E, lam, Er = O.gsvd(K, R)
    I = np.eye(M)
    EH = np.conj(np.swapaxes(E, 1, 2))
    ErH = np.conj(np.swapaxes(Er, 1, 2))
    assert np.abs(np.matmul(EH, E) - I).max() < 1e-12
    assert np.abs(np.matmul(ErH, Er) - I).max() < 1e-12
    rec = np.matmul(E * lam[:, None, :], ErH)
    assert np.linalg.norm(rec - A) <= 1e-12 * np.linalg.norm(A)
    assert np.all(lam >= 0) and np.all(np.diff(lam, axis=1) <= 0)
    # A is K^{-1} R (not R K^{-1}, not K R).
    assert np.linalg.norm(np.matmul(K, A) - R) <= 1e-11 * np.linalg.norm(R)
    # Left vectors: A A^H e_i = lam_i^2 e_i, lam^2 = eigenvalues of A A^H.
    AAH = np.matmul(A, np.conj(np.swapaxes(A, 1, 2)))
    w = np.linalg.eigvalsh(AAH)[:, ::-1]
    assert np.allclose(lam ** 2, w, rtol=1e-9, atol=1e-12 * w.max())
    for b in range(B):
        for i in range(M):
            v = AAH[b] @ E[b, :, i]
            assert np.linalg.norm(v - lam[b, i] ** 2 * E[b, :, i]) <= 1e-9 * lam[b, 0] ** 2
            # and A^H e_i = lam_i er_i
            u = np.conj(A[b]).T @ E[b, :, i]
            assert np.linalg.norm(u - lam[b, i] * Er[b, :, i]) <= 1e-9 * lam[b, 0]


def pin_gsvd_closed_forms(O):
    rng = np.random.default_rng(15)
    # M = 2: sigma^2 = (F +- sqrt(F^2 - 4 |det A|^2)) / 2, F = ||A||_F^2.
    for _ in range(5):
        A = _crand(rng, 2, 2)
        F = np.sum(np.abs(A) ** 2)
        dt = abs(np.linalg.det(A))
        disc = np.sqrt(F * F - 4 * dt * dt)
        s2 = np.array([(F + disc) / 2, (F - disc) / 2])
        _, _, lam, _ = O.gsvd(np.eye(2)[None].astype(complex), A[None])
        assert np.allclose(lam[0] ** 2, s2, rtol=1e-10)
    # M = 2..4: sigma^2 are the roots of the characteristic polynomial of A A^H.
    for M in (2, 3, 4):
        K = _herm_pd(rng, 1, M, cond=5.0)
        R = O.correlation(_crand(rng, 9, 1, M))
        A, _, lam, _ = O.gsvd(K, R)
        AAH = A[0] @ np.conj(A[0]).T
        r = np.sort(np.real(np.roots(_faddeev_leverrier(AAH))))[::-1]
        assert np.allclose(lam[0] ** 2, r, rtol=1e-7, atol=1e-12)


def pin_k_identity_reduces_to_sevd(O):
    """K = I: GSVD-MUSIC is SEVD-MUSIC (Sec. II, Sec. IV-B): the left singular
    vectors are eigenvectors of R and the singular values its eigenvalues."""
    rng = np.random.default_rng(16)
    B, M, Ns = 4, 6, 2
    R = O.correlation(_crand(rng, 12, B, M))
    I = np.broadcast_to(np.eye(M), (B, M, M)).astype(complex)
    _, E, lam, _ = O.gsvd(I, R)
    w, V = np.linalg.eigh(R)
    w, V = w[:, ::-1], V[:, :, ::-1]
    assert np.allclose(lam, w, rtol=1e-10, atol=1e-12)
    En = O.noise_subspace(E, Ns)
    Vn = V[:, :, Ns:]
    P1 = np.matmul(En, np.conj(np.swapaxes(En, 1, 2)))
    P2 = np.matmul(Vn, np.conj(np.swapaxes(Vn, 1, 2)))
    assert np.abs(P1 - P2).max() < 1e-10


# --------------------------------------------------------------------------
# spectrum (eq. 5), bin sum (eq. 6)
# --------------------------------------------------------------------------

def pin_spectrum_golden(O):
    for r in _lines("spectrum_hand.txt"):
        M, Ns = int(r[1]), int(r[2])
        bar = [i for i, t in enumerate(r) if t == "|"]
        Rv = np.array(r[3:bar[0]], float)
        hv = np.array(r[bar[0] + 1:bar[1]], float)
        pa, ps = float(r[bar[1] + 1]), float(r[bar[1] + 2])
        R = (Rv[0::2] + 1j * Rv[1::2]).reshape(1, M, M)
        h = (hv[0::2] + 1j * hv[1::2]).reshape(1, 1, M)
        I = np.eye(M)[None].astype(complex)
        _, E, _, _ = O.gsvd(I, R)
        En = O.noise_subspace(E, Ns)
        assert abs(O.spectrum(h, En, "abs")[0, 0] - pa) < 1e-12
        assert abs(O.spectrum(h, En, "sq")[0, 0] - ps) < 1e-12


def pin_spectrum_closed_form(O):
    """K = I, R = s a a^H + sigma^2 I, Ns = 1: E_n E_n^H = I - a a^H / ||a||^2,
    so P_sq(h) = ||h||^2 / (||h||^2 - |h^H a|^2 / ||a||^2) for every h."""
    rng = np.random.default_rng(17)
    M = 6
    a = _crand(rng, M)
    R = (3.0 * np.outer(a, a.conj()) + 0.5 * np.eye(M))[None]
    I = np.eye(M)[None].astype(complex)
    _, E, _, _ = O.gsvd(I, R)
    En = O.noise_subspace(E, 1)
    H = _crand(rng, 1, 40, M)
    P = O.spectrum(H, En, "sq")[0]
    hh = np.sum(np.abs(H[0]) ** 2, axis=1)
    ha = np.abs(H[0] @ a.conj()) ** 2 / np.vdot(a, a).real
    assert np.allclose(P, hh / (hh - ha), rtol=1e-10)


def pin_plane_wave_orthogonal(O):
    """A noiseless plane wave with K = c I lies orthogonal to the noise
    subspace, so its direction is where the spectrum peaks (Sec. III-A)."""
    w = synth.uca8_single_source(seed=3, nblk=1, snr_db=0.0)
    d0 = int(w.src_grid_idx[0, 0])
    assert d0 >= 0
    B, M = w.B, w.M
    rng = np.random.default_rng(5)
    h0 = w.H[:, d0, :]  # [B][M]
    S = _crand(rng, w.T, B)
    X = h0[None, :, :] * S[:, :, None]
    K = 2.0 * np.broadcast_to(np.eye(M), (B, M, M)).astype(complex)
    R = O.correlation(X)
    _, E, _, _ = O.gsvd(K, R)
    En = O.noise_subspace(E, 1)
    proj = np.abs(np.einsum("bm,bmi->bi", np.conj(h0), En))
    assert proj.max() < 1e-9 * np.sqrt(M)
    # Add weak white noise so that the spectrum stays finite; argmax = source.
    X2 = X + 1e-3 * _crand(rng, w.T, B, M)
    for form in ("abs", "sq"):
        out = O.localize_block(X2, K, w.H, 1, w.grid.n_az, w.grid.n_el, form)
        assert int(out["idx"][0]) == d0
        assert int(np.argmax(out["Pbar"])) == d0


def pin_invariances(O):
    rng = np.random.default_rng(18)
    B, M, T, D, Ns = 3, 5, 20, 9, 2
    X = _crand(rng, T, B, M)
    K = _herm_pd(rng, B, M, cond=20.0)
    H = _crand(rng, B, D, M)

    def P_of(X_, K_, H_, form):
        R = O.correlation(X_)
        _, E, _, _ = O.gsvd(K_, R)
        return O.spectrum(H_, O.noise_subspace(E, Ns), form)

    for form in ("abs", "sq"):
        P0 = P_of(X, K, H, form)
        perm = rng.permutation(M)
        P1 = P_of(X[..., perm], K[:, perm][:, :, perm], H[..., perm], form)
        assert np.allclose(P0, P1, rtol=1e-9)
        ph = np.exp(1j * rng.uniform(0, 2 * np.pi, (B, M)))
        Dm = ph[:, :, None] * np.eye(M)[None]
        K2 = np.matmul(np.matmul(Dm, K), np.conj(np.swapaxes(Dm, 1, 2)))
        P2 = P_of(X * ph[None], K2, H * ph[:, None, :], form)
        assert np.allclose(P0, P2, rtol=1e-9)
        P3 = P_of(3.0 * X, 0.25 * K, H, form)
        assert np.allclose(P0, P3, rtol=1e-9)


def pin_bin_sum(O):
    rng = np.random.default_rng(19)
    B, D = 7, 11
    assert np.allclose(O.bin_sum(np.ones((B, D))), np.full(D, float(B)))
    P1, P2 = rng.random((B, D)), rng.random((B, D))
    assert np.allclose(O.bin_sum(P1 + 2 * P2), O.bin_sum(P1) + 2 * O.bin_sum(P2))
    # Each bin contributes to its own direction only.
    E = np.zeros((B, D))
    E[3, 5] = 1.0
    s = O.bin_sum(E)
    assert s[5] == 1.0 and np.count_nonzero(s) == 1


# --------------------------------------------------------------------------
# peaks
# --------------------------------------------------------------------------

def pin_peaks_golden(O):
    for r in _lines("peaks_hand.txt"):
        bar = [i for i, t in enumerate(r) if t == "|"]
        n_az, n_el, Ns = int(r[0]), int(r[1]), int(r[2])
        Pbar = np.array(r[bar[0] + 1:bar[1]], float)
        idx = np.array(r[bar[1] + 1:bar[2]], int)
        val = np.array(r[bar[2] + 1:], float)
        i2, v2 = O.peaks(Pbar, n_az, n_el, Ns)
        assert list(i2) == list(idx)
        assert np.allclose(v2, val)


def pin_peaks_bruteforce(O):
    """Random small grids: the selection equals an independent sort of all
    grid points that beat every neighbour (tie rule on index)."""
    rng = np.random.default_rng(20)
    for trial in range(30):
        n_az, n_el = int(rng.integers(3, 9)), int(rng.integers(1, 5))
        D = n_az * n_el
        Pbar = rng.integers(0, 4, D).astype(float)  # many ties
        Ns = int(rng.integers(1, 5))
        grid = Pbar.reshape(n_el, n_az)
        pk = []
        for e in range(n_el):
            for a in range(n_az):
                d = e * n_az + a
                nb = set()
                for ee in (e - 1, e, e + 1):
                    if 0 <= ee < n_el:
                        for aa in (a - 1, a, a + 1):
                            nb.add(ee * n_az + aa % n_az)
                nb.discard(d)
                if all((grid.flat[d], -d) > (grid.flat[n], -n) for n in nb):
                    pk.append(d)
        pk.sort(key=lambda d: (-Pbar[d], d))
        exp = (pk + [-1] * Ns)[:Ns]
        i2, _ = O.peaks(Pbar, n_az, n_el, Ns)
        assert list(i2) == exp, (trial, n_az, n_el, Ns)


def pin_peaks_range_golden(O):
    """Hand-derived search ranges (Sec. III-A, last step): grids with the range
    across the azimuth wrap, an in-range direction beaten by an out-of-range
    neighbour, and a direction set whose only peak lies outside the range."""
    for r in _lines("peaks_range_hand.txt"):
        bar = [i for i, t in enumerate(r) if t == "|"]
        if r[0] == "grid":
            n_az, n_el, Ns = int(r[1]), int(r[2]), int(r[3])
            Pbar = np.array(r[bar[0] + 1:bar[1]], float)
            mask = np.array(r[bar[1] + 1:bar[2]], int).astype(bool)
            idx = np.array(r[bar[2] + 1:bar[3]], int)
            val = np.array(r[bar[3] + 1:], float)
            i2, v2 = O.peaks(Pbar, n_az, n_el, Ns, mask)
        else:
            D, Ns = int(r[1]), int(r[2])
            Pbar = np.array(r[bar[0] + 1:bar[1]], float)
            ptr = np.array(r[bar[1] + 1:bar[2]], int)
            nbr = np.array(r[bar[2] + 1:bar[3]], int)
            mask = np.array(r[bar[3] + 1:bar[4]], int).astype(bool)
            idx = np.array(r[bar[4] + 1:bar[5]], int)
            val = np.array(r[bar[5] + 1:], float)
            assert Pbar.size == D and mask.size == D
            i2, v2 = O.peaks_nbr(Pbar, ptr, nbr, Ns, mask)
        assert list(i2) == list(idx), (r, list(i2))
        assert np.allclose(v2, val)


def pin_peaks_range_bruteforce(O):
    """Random grids and ranges: the selection is the independent brute-force
    peak set (every neighbour counts) cut to the range, sorted; the full range
    equals no range; an empty range reports nothing."""
    rng = np.random.default_rng(23)
    for trial in range(30):
        n_az, n_el = int(rng.integers(3, 9)), int(rng.integers(1, 5))
        D = n_az * n_el
        Pbar = rng.integers(0, 5, D).astype(float)
        Ns = int(rng.integers(1, 5))
        mask = rng.random(D) < 0.5
        pk = []
        for e in range(n_el):
            for a in range(n_az):
                d = e * n_az + a
                nb = {ee * n_az + aa % n_az for ee in (e - 1, e, e + 1) if 0 <= ee < n_el
                      for aa in (a - 1, a, a + 1)} - {d}
                if mask[d] and all((Pbar[d], -d) > (Pbar[n], -n) for n in nb):
                    pk.append(d)
        pk.sort(key=lambda d: (-Pbar[d], d))
        i2, v2 = O.peaks(Pbar, n_az, n_el, Ns, mask)
        assert list(i2) == (pk + [-1] * Ns)[:Ns], (trial, n_az, n_el)
        full = O.peaks(Pbar, n_az, n_el, Ns, np.ones(D, bool))
        none = O.peaks(Pbar, n_az, n_el, Ns)
        assert list(full[0]) == list(none[0])
        empty = O.peaks(Pbar, n_az, n_el, Ns, np.zeros(D, bool))
        assert list(empty[0]) == [-1] * Ns and not np.any(empty[1])


def pin_peaks_nbr_golden(O):
    for r in _lines("peaks_nbr_hand.txt"):
        bar = [i for i, t in enumerate(r) if t == "|"]
        D, Ns = int(r[0]), int(r[1])
        Pbar = np.array(r[bar[0] + 1:bar[1]], float)
        ptr = np.array(r[bar[1] + 1:bar[2]], int)
        nbr = np.array(r[bar[2] + 1:bar[3]], int)
        idx = np.array(r[bar[3] + 1:bar[4]], int)
        val = np.array(r[bar[4] + 1:], float)
        assert Pbar.size == D and ptr.size == D + 1
        i2, v2 = O.peaks_nbr(Pbar, ptr, nbr, Ns)
        assert list(i2) == list(idx)
        assert np.allclose(v2, val)


def pin_peaks_nbr_is_the_grid_rule_on_grids(O):
    """With the grid's 8-neighbourhood as lists, the list rule selects
    exactly what the (separately pinned) grid rule selects, ties included,
    and the peak margins agree."""
    from paper_2504_03373_gb300 import synth
    rng = np.random.default_rng(21)
    shapes = [(72, 19), (6, 3), (8, 1), (1, 1), (5, 7), (3, 2)]
    for trial in range(24):
        n_az, n_el = shapes[trial % len(shapes)]
        D = n_az * n_el
        Pbar = rng.integers(0, 4, D).astype(float) if trial % 2 else rng.random(D)
        Ns = int(rng.integers(1, 6))
        ptr, nbr = synth.grid_neighbours(n_az, n_el)
        i1, v1 = O.peaks(Pbar, n_az, n_el, Ns)
        i2, v2 = O.peaks_nbr(Pbar, ptr, nbr, Ns)
        assert list(i1) == list(i2), (trial, n_az, n_el)
        assert np.array_equal(v1, v2)
        m1 = O.peak_margin(Pbar, n_az, n_el, Ns)
        m2 = O.peak_margin_nbr(Pbar, ptr, nbr, Ns)
        assert m1 == m2 or (np.isinf(m1) and np.isinf(m2)), (trial, m1, m2)


def pin_peaks_nbr_relabelling(O):
    """Renaming the directions (a permutation applied to the values and to
    the neighbour lists) renames the selected peaks, for distinct values on a
    random symmetric neighbour graph."""
    rng = np.random.default_rng(22)
    for trial in range(10):
        D = int(rng.integers(5, 40))
        sets = [set() for _ in range(D)]
        for _ in range(2 * D):
            a, b = rng.integers(0, D, 2)
            if a != b:
                sets[a].add(int(b))
                sets[b].add(int(a))
        ptr = np.zeros(D + 1, int)
        ptr[1:] = np.cumsum([len(x) for x in sets])
        nbr = np.array([n for x in sets for n in sorted(x)], int)
        Pbar = rng.permutation(D).astype(float) + 1.0  # distinct
        Ns = int(rng.integers(1, 5))
        perm = rng.permutation(D)  # old d -> new perm[d]
        inv = np.argsort(perm)
        sets2 = [{int(perm[n]) for n in sets[inv[d2]]} for d2 in range(D)]
        ptr2 = np.zeros(D + 1, int)
        ptr2[1:] = np.cumsum([len(x) for x in sets2])
        nbr2 = np.array([n for x in sets2 for n in sorted(x)], int)
        P2 = Pbar[inv]
        i1, v1 = O.peaks_nbr(Pbar, ptr, nbr, Ns)
        i2, v2 = O.peaks_nbr(P2, ptr2, nbr2, Ns)
        assert [int(perm[d]) if d >= 0 else -1 for d in i1] == list(i2)
        assert np.array_equal(v1, v2)


def pin_sevd(O):
    """R = E diag(lam) E^H with E unitary and lam descending; the 2x2 case
    against the closed-form eigenvalues (tr/2 +- sqrt((tr/2)^2 - det))."""
    rng = np.random.default_rng(61)
    for M in (2, 3, 7):
        X = _crand(rng, 4, M, 2 * M)
        R = np.matmul(X, np.conj(np.swapaxes(X, -1, -2))) / (2 * M)
        E, lam = O.sevd(R)
        EH = np.conj(np.swapaxes(E, -1, -2))
        assert np.abs(np.matmul(EH, E) - np.eye(M)).max() < 1e-12
        rec = np.matmul(E * lam[..., None, :], EH)
        assert np.abs(rec - R).max() < 1e-12 * np.abs(R).max()
        assert np.all(np.diff(lam, axis=-1) <= 1e-12)
        if M == 2:
            tr = np.real(R[:, 0, 0] + R[:, 1, 1])
            det = np.real(R[:, 0, 0] * R[:, 1, 1] - R[:, 0, 1] * R[:, 1, 0])
            disc = np.sqrt((tr / 2) ** 2 - det)
            assert np.allclose(lam[:, 0], tr / 2 + disc, rtol=1e-12)
            assert np.allclose(lam[:, 1], tr / 2 - disc, rtol=1e-12)


def pin_gevd(O):
    """R E = K E diag(lam), E^H K E = I, lam descending; K = I gives the
    SEVD eigenvalues; the 2x2 case against the roots of det(R - lam K) = 0;
    under R = s a a^H + sigma^2 K the noise eigenvalues equal sigma^2 and
    their eigenvectors are exactly orthogonal to a (the GEVD-MUSIC model)."""
    rng = np.random.default_rng(62)
    for M in (2, 3, 6):
        K = _herm_pd(rng, 3, M, cond=50.0)
        X = _crand(rng, 3, M, 2 * M)
        R = np.matmul(X, np.conj(np.swapaxes(X, -1, -2))) / (2 * M)
        E, lam = O.gevd(K, R)
        EH = np.conj(np.swapaxes(E, -1, -2))
        assert np.abs(np.matmul(EH, np.matmul(K, E)) - np.eye(M)).max() < 1e-10
        res = np.matmul(R, E) - np.matmul(K, E) * lam[..., None, :]
        assert np.abs(res).max() < 1e-10 * np.abs(R).max()
        assert np.all(np.diff(lam, axis=-1) <= 1e-12)
        _, lam_i = O.gevd(np.broadcast_to(np.eye(M), R.shape).astype(complex), R)
        assert np.allclose(lam_i, np.linalg.eigvalsh(R)[..., ::-1], rtol=1e-10, atol=1e-12)
        if M == 2:
            # det(R - l K) = a l^2 + b l + c
            a = np.real(K[:, 0, 0] * K[:, 1, 1] - K[:, 0, 1] * K[:, 1, 0])
            b = -np.real(R[:, 0, 0] * K[:, 1, 1] + K[:, 0, 0] * R[:, 1, 1]
                         - R[:, 0, 1] * K[:, 1, 0] - K[:, 0, 1] * R[:, 1, 0])
            c = np.real(R[:, 0, 0] * R[:, 1, 1] - R[:, 0, 1] * R[:, 1, 0])
            disc = np.sqrt(b * b - 4 * a * c)
            assert np.allclose(lam[:, 0], (-b + disc) / (2 * a), rtol=1e-10)
            assert np.allclose(lam[:, 1], (-b - disc) / (2 * a), rtol=1e-10)
    M, sigma2, s = 8, 0.3, 5.0
    K = _herm_pd(rng, 1, M, cond=1e3)
    a_vec = np.exp(1j * rng.uniform(0, 2 * np.pi, M))
    R = s * np.outer(a_vec, np.conj(a_vec))[None] + sigma2 * K
    E, lam = O.gevd(K, R)
    assert np.allclose(lam[0, 1:], sigma2, rtol=1e-9)
    assert np.abs(np.conj(a_vec) @ E[0][:, 1:]).max() < 1e-9


# --------------------------------------------------------------------------
# test gating: peak margin and noise-value gap (they decide where the GPU
# tests grade peak indices and individual noise vectors)
# --------------------------------------------------------------------------

def pin_peak_margin(O):
    """Hand-computed margins: (a) lead of the Ns-th selected peak over the
    best unselected one and (b) each selected peak's lead over its largest
    neighbour, both relative to the peak."""
    row = np.array([1, 5, 2, 1, 1, 4, 1, 1], float)  # one elevation, azimuth wraps
    # Ns = 1: peaks at 1 (5) and 5 (4); (a) (5 - 4) / 5, (b) (5 - 2) / 5
    assert np.isclose(O.peak_margin(row, 8, 1, 1), 0.2)
    # Ns = 2: nothing left unselected; (b) min((5 - 2) / 5, (4 - 1) / 4)
    assert np.isclose(O.peak_margin(row, 8, 1, 2), 0.6)
    assert np.isclose(O.peak_margin(row, 8, 1, 3), 0.6)  # fewer peaks than Ns
    # A plateau has no robust peak.
    assert O.peak_margin(np.full(10, 3.0), 5, 2, 1) == 0.0
    # 4 azimuths x 3 elevations: 10 at (el 1, az 2), its diagonal neighbour
    # (el 2, az 3) 9, the rest 1 (whose lowest index is a grid peak):
    # min((10 - 1) / 10, (10 - 9) / 10)
    g = np.ones(12)
    g[1 * 4 + 2] = 10.0
    g[2 * 4 + 3] = 9.0
    assert np.isclose(O.peak_margin(g, 4, 3, 1), 0.1)
    # Positive scaling leaves the relative margin unchanged.
    assert np.isclose(O.peak_margin(7.5 * g, 4, 3, 1), 0.1)


def pin_noise_gap(O):
    """Smallest relative gap between consecutive noise values, per bin."""
    assert np.isclose(O.noise_gap(np.array([10.0, 5, 4, 2, 1]), 2), 0.5)
    assert O.noise_gap(np.array([9.0, 3, 3, 1]), 1) == 0.0  # repeated noise value
    assert np.isinf(O.noise_gap(np.array([7.0, 2]), 1))     # one noise value
    lam = np.array([[10.0, 5, 4, 2, 1], [10.0, 8, 4, 2, 1]])
    assert np.allclose(O.noise_gap(lam, 1), [0.2, 0.5])
    assert O.noise_gap(np.array([1.0, 0, 0]), 1) == 0.0      # null space


ALL_PINS = [
    pin_correlation_golden,
    pin_correlation_bruteforce,
    pin_correlation_structure,
    pin_whiten_golden,
    pin_whiten_solves,
    pin_gsvd_golden,
    pin_gsvd_factorisation,
    pin_gsvd_closed_forms,
    pin_k_identity_reduces_to_sevd,
    pin_spectrum_golden,
    pin_spectrum_closed_form,
    pin_plane_wave_orthogonal,
    pin_invariances,
    pin_bin_sum,
    pin_peaks_golden,
    pin_peaks_bruteforce,
    pin_peaks_nbr_golden,
    pin_peaks_nbr_is_the_grid_rule_on_grids,
    pin_peaks_nbr_relabelling,
    pin_peaks_range_golden,
    pin_peaks_range_bruteforce,
    pin_sevd,
    pin_gevd,
    pin_peak_margin,
    pin_noise_gap,
]
