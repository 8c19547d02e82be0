"""FP64 CPU oracle of the GSVD-MUSIC localization hot path.

TEST INFRASTRUCTURE ONLY.  Only the test suite, the package's smoke check and
the CPU-baseline leg of the benchmark may import this module.  The product
path never calls it, and it shares no code with the CUDA library.

Each function restates one step of the method of Lin et al., "An Efficient
GPU-based Implementation for Noise Robust Sound Source Localization"
(arXiv 2504.03373), Sec. III-A, as plain NumPy in complex128 / float64:

  correlation      eq. 2-3   R = (1/T) sum_f X X^H over one block of T frames
  whiten           eq. 4, Sec. III-B   A = K^{-1} R by Gaussian elimination
  gsvd             eq. 4     A = E Lambda E_r^H, singular values descending
  sevd, gevd       Sec. II   the SEVD (K = I) and GEVD (R e = lam K e) variants
  noise_subspace   Sec. III-A (E_n)    columns Ns+1..M of E
  spectrum         eq. 5     P = |h^H h| / sum_i |h^H e_i|  (and squared form)
  bin_sum          eq. 6     Pbar = sum over bins of P
  peaks            Sec. III-A (peak search)   grid local maxima, top Ns
  peaks_nbr        Sec. III-A (peak search)   the same rule over an arbitrary
                   direction set whose neighbours are given as lists (the
                   paper's measured transfer functions cover 2522 directions
                   over the sphere, Sec. V, which form no grid)

Readings of the paper where it is silent or garbled (they are the same
readings the CUDA path implements):

* eq. 2 prints X X^*; the text defines (.)^H and calls R positive
  semi-definite, so R_ins = X X^H, i.e. R_ij = x_i conj(x_j).
* eq. 3 is read block-wise: one R per non-overlapping block of T frames
  (the paper processes "at fixed intervals", Sec. VI).
* eq. 4: E has the left singular vectors as columns; Lambda is real,
  non-negative and descending; the decomposition is the plain SVD of the
  non-Hermitian product K^{-1} R.
* eq. 5 sums over i but prints e_n and no square.  ``form='abs'`` is the
  literal reading sum_i |h^H e_i|; ``form='sq'`` is sum_i |h^H e_i|^2, the
  textbook MUSIC denominator, which does not depend on the basis chosen
  inside the noise subspace.  A zero denominator is clamped to 1e-300.
* eq. 6 is a sum over bins (not a mean).
* Peak search (no rule given): on an n_el x n_az grid, d = e * n_az + a,
  azimuth neighbours wrap, elevation neighbours outside the grid are dropped,
  8-neighbourhood.  d is a peak iff for every neighbour n,
  Pbar[d] > Pbar[n] or (Pbar[d] == Pbar[n] and d < n).  Peaks are ranked by
  value descending, ties by lower d; the first Ns are returned, padded with
  index -1 / value 0.
* Peak search over a direction set that is not a grid: the neighbours of d
  are given as a list (compressed rows: nbr_idx[nbr_ptr[d]:nbr_ptr[d + 1]]);
  d is a peak iff for every listed neighbour n != d the same comparison
  holds; ranking and padding as on the grid.  The grid rule is this rule with
  the 8-neighbourhood lists.
* The search range [theta_min, theta_max] (Sec. III-A, last step) is a set of
  directions, given as a boolean mask over the D directions (None: all of
  them).  Only directions inside the range may be reported as peaks; the
  peak test of such a direction still compares it with all of its
  neighbours, inside the range or not, since the spectrum exists everywhere.
"""

from __future__ import annotations

import numpy as np

DEN_FLOOR = 1e-300


def correlation(X: np.ndarray) -> np.ndarray:
    """eq. 2-3: X [T][B][M] -> R [B][M][M], R = (1/T) sum_f x_f x_f^H."""
    X = np.asarray(X, dtype=np.complex128)
    T = X.shape[0]
    return np.einsum("tbi,tbj->bij", X, np.conj(X)) / T


def whiten(K: np.ndarray, R: np.ndarray) -> np.ndarray:
    """eq. 4 (Sec. III-B): A = K^{-1} R, with K^{-1} applied by Gaussian
    elimination (LU with partial pivoting), per bin."""
    K = np.asarray(K, dtype=np.complex128)
    R = np.asarray(R, dtype=np.complex128)
    return np.linalg.solve(K, R)


def inverse_by_cholesky(K: np.ndarray) -> np.ndarray:
    """K^{-1} = L^{-H} L^{-1} with K = L L^H (the factorisation the GPU uses
    for the preset noise correlation).  Used by tests to check that both
    routes give the same A."""
    K = np.asarray(K, dtype=np.complex128)
    L = np.linalg.cholesky(K)
    I = np.broadcast_to(np.eye(K.shape[-1]), K.shape)
    Linv = np.linalg.solve(L, I)
    return np.matmul(np.conj(np.swapaxes(Linv, -1, -2)), Linv)


def gsvd(K: np.ndarray, R: np.ndarray):
    """eq. 4: K^{-1} R = E Lambda E_r^H.

    Returns (A, E, lam, Er): E [B][M][M] with the left singular vectors as
    columns, lam [B][M] descending and non-negative, Er [B][M][M] the right
    singular vectors as columns.
    """
    A = whiten(K, R)
    U, s, Vh = np.linalg.svd(A)
    return A, U, s, np.conj(np.swapaxes(Vh, -1, -2))


def sevd(R: np.ndarray):
    """SEVD-MUSIC's decomposition (Sec. II; eq. 4 with K = I): the Hermitian
    eigendecomposition R = E diag(lam) E^H.  Returns (E, lam), eigenvalues
    descending, eigenvectors as columns of E."""
    lam, E = np.linalg.eigh(np.asarray(R, dtype=np.complex128))
    return E[..., ::-1], lam[..., ::-1]


def gevd(K: np.ndarray, R: np.ndarray):
    """The generalised eigenproblem of the pair (R, K), R e = lam K e (the
    GEVD that Sec. II contrasts with the GSVD), by Cholesky reduction: with
    K = L L^H the Hermitian matrix L^{-1} R L^{-H} has the same eigenvalues,
    and its eigenvectors y give e = L^{-H} y.  Returns (E, lam): eigenvalues
    descending, columns of E K-orthonormal (E^H K E = I)."""
    K = np.asarray(K, dtype=np.complex128)
    R = np.asarray(R, dtype=np.complex128)
    L = np.linalg.cholesky(K)
    Linv = np.linalg.inv(L)
    LinvH = np.conj(np.swapaxes(Linv, -1, -2))
    lam, Y = np.linalg.eigh(np.matmul(np.matmul(Linv, R), LinvH))
    E = np.matmul(LinvH, Y)
    return E[..., ::-1], lam[..., ::-1]


def noise_subspace(E: np.ndarray, Ns: int) -> np.ndarray:
    """E_n = [e_{Ns+1} ... e_M] (the non-zero columns of E_n, Sec. III-A)."""
    return E[..., :, Ns:]


def spectrum(H: np.ndarray, En: np.ndarray, form: str = "abs") -> np.ndarray:
    """eq. 5 for every (bin, direction).

    H [B][D][M] steering vectors, En [B][M][M-Ns] -> P [B][D].
    """
    H = np.asarray(H, dtype=np.complex128)
    Y = np.matmul(np.conj(H), En)  # [B][D][M-Ns], Y_di = h_d^H e_i
    num = np.real(np.sum(np.conj(H) * H, axis=-1))  # |h^H h|
    if form == "abs":
        den = np.sum(np.abs(Y), axis=-1)
    elif form == "sq":
        den = np.sum(np.abs(Y) ** 2, axis=-1)
    else:
        raise ValueError(form)
    return num / np.maximum(den, DEN_FLOOR)


def bin_sum(P: np.ndarray) -> np.ndarray:
    """eq. 6: Pbar [D] = sum over bins of P [B][D]."""
    return np.sum(P, axis=-2)


def is_peak(Pbar: np.ndarray, n_az: int, n_el: int) -> np.ndarray:
    """Boolean [D]: the grid peak rule stated in the module docstring."""
    Pbar = np.asarray(Pbar)
    D = n_az * n_el
    assert Pbar.shape == (D,)
    out = np.zeros(D, dtype=bool)
    for d in range(D):
        e, a = divmod(d, n_az)
        ok = True
        for de in (-1, 0, 1):
            ee = e + de
            if ee < 0 or ee >= n_el:
                continue
            for da in (-1, 0, 1):
                if de == 0 and da == 0:
                    continue
                n = ee * n_az + (a + da) % n_az
                if n == d:
                    continue
                if Pbar[d] > Pbar[n] or (Pbar[d] == Pbar[n] and d < n):
                    continue
                ok = False
                break
            if not ok:
                break
        out[d] = ok
    return out


def _in_range(cand: np.ndarray, mask) -> np.ndarray:
    """The candidate peaks inside the search range (mask: bool [D] or None)."""
    if mask is None:
        return cand
    mask = np.asarray(mask, dtype=bool)
    return np.asarray([d for d in cand if mask[d]], dtype=np.int64)


def peaks(Pbar: np.ndarray, n_az: int, n_el: int, Ns: int, mask=None):
    """Peak search over [theta_min, theta_max] (mask; None: the whole grid):
    the Ns largest grid peaks inside the range, ties to the lower index.
    Returns (idx, val)."""
    Pbar = np.asarray(Pbar, dtype=np.float64)
    cand = _in_range(np.nonzero(is_peak(Pbar, n_az, n_el))[0], mask)
    order = sorted(cand.tolist(), key=lambda d: (-Pbar[d], d))
    idx = np.full(Ns, -1, dtype=np.int64)
    val = np.zeros(Ns, dtype=np.float64)
    for k, d in enumerate(order[:Ns]):
        idx[k] = d
        val[k] = Pbar[d]
    return idx, val


def is_peak_nbr(Pbar: np.ndarray, nbr_ptr: np.ndarray, nbr_idx: np.ndarray) -> np.ndarray:
    """Boolean [D]: d is a peak iff Pbar[d] > Pbar[n], or they are equal and
    d < n, for every listed neighbour n of d (n == d is skipped)."""
    Pbar = np.asarray(Pbar)
    D = Pbar.shape[0]
    out = np.zeros(D, dtype=bool)
    for d in range(D):
        ok = True
        for n in nbr_idx[nbr_ptr[d]:nbr_ptr[d + 1]]:
            n = int(n)
            if n == d:
                continue
            if not (Pbar[d] > Pbar[n] or (Pbar[d] == Pbar[n] and d < n)):
                ok = False
                break
        out[d] = ok
    return out


def peaks_nbr(Pbar: np.ndarray, nbr_ptr: np.ndarray, nbr_idx: np.ndarray, Ns: int, mask=None):
    """Peak search over a direction set with neighbour lists: the Ns largest
    peaks (is_peak_nbr) inside the search range (mask; None: all),
    ties to the lower index.  Returns (idx, val)."""
    Pbar = np.asarray(Pbar, dtype=np.float64)
    cand = _in_range(np.nonzero(is_peak_nbr(Pbar, nbr_ptr, nbr_idx))[0], mask)
    order = sorted(cand.tolist(), key=lambda d: (-Pbar[d], d))
    idx = np.full(Ns, -1, dtype=np.int64)
    val = np.zeros(Ns, dtype=np.float64)
    for k, d in enumerate(order[:Ns]):
        idx[k] = d
        val[k] = Pbar[d]
    return idx, val


def peak_margin_nbr(Pbar: np.ndarray, nbr_ptr: np.ndarray, nbr_idx: np.ndarray,
                    Ns: int, mask=None) -> float:
    """peak_margin over a direction set with neighbour lists."""
    Pbar = np.asarray(Pbar, dtype=np.float64)
    idx, _ = peaks_nbr(Pbar, nbr_ptr, nbr_idx, Ns, mask)
    sel = [int(d) for d in idx if d >= 0]
    if not sel:
        return 0.0
    cand = _in_range(np.nonzero(is_peak_nbr(Pbar, nbr_ptr, nbr_idx))[0], mask)
    rest = [Pbar[d] for d in cand if d not in sel]
    low = Pbar[sel[-1]]
    margin = (low - max(rest)) / abs(low) if rest else np.inf
    for d in sel:
        nb = [Pbar[int(n)] for n in nbr_idx[nbr_ptr[d]:nbr_ptr[d + 1]] if int(n) != d]
        if nb:
            margin = min(margin, (Pbar[d] - max(nb)) / abs(Pbar[d]))
    return float(margin)


def peak_margin(Pbar: np.ndarray, n_az: int, n_el: int, Ns: int, mask=None) -> float:
    """Relative robustness of the peak search: the smaller of
    (a) the Ns-th selected peak's lead over the best unselected peak inside
    the search range and (b) each selected peak's lead over its own largest
    neighbour, each divided by the peak's value.  Peak indices are graded
    only where this margin exceeds the compared path's tolerance."""
    Pbar = np.asarray(Pbar, dtype=np.float64)
    idx, _ = peaks(Pbar, n_az, n_el, Ns, mask)
    sel = [int(d) for d in idx if d >= 0]
    if not sel:
        return 0.0
    cand = _in_range(np.nonzero(is_peak(Pbar, n_az, n_el))[0], mask)
    rest = [Pbar[d] for d in cand if d not in sel]
    low = Pbar[sel[-1]]
    margin = (low - max(rest)) / abs(low) if rest else np.inf
    for d in sel:
        e, a = divmod(d, n_az)
        nb = -np.inf
        for de in (-1, 0, 1):
            ee = e + de
            if ee < 0 or ee >= n_el:
                continue
            for da in (-1, 0, 1):
                n = ee * n_az + (a + da) % n_az
                if n != d:
                    nb = max(nb, Pbar[n])
        if np.isfinite(nb):
            margin = min(margin, (Pbar[d] - nb) / abs(Pbar[d]))
    return float(margin)


def noise_gap(lam: np.ndarray, Ns: int) -> np.ndarray:
    """Smallest relative gap between consecutive noise singular values
    (lam_{Ns+1..M}) per bin; 0 where the noise subspace has a (near) repeated
    value, i.e. where individual noise vectors are not determined."""
    lam = np.asarray(lam, dtype=np.float64)
    ln = lam[..., Ns:]
    if ln.shape[-1] < 2:
        return np.full(lam.shape[:-1], np.inf)
    g = (ln[..., :-1] - ln[..., 1:]) / np.maximum(ln[..., :-1], DEN_FLOOR)
    return np.min(g, axis=-1)


def localize_block(X, K, H, Ns, n_az, n_el, form="abs", nbr=None, mask=None):
    """The whole hot path for one block: X [T][B][M], K [B][M][M],
    H [B][D][M] -> dict with R, A, E, lam, P, Pbar, idx, val.  nbr =
    (nbr_ptr, nbr_idx): peak search over those neighbour lists instead of
    the n_el x n_az grid; mask: the search range (bool [D], None: all)."""
    R = correlation(X)
    A, E, lam, _ = gsvd(K, R)
    En = noise_subspace(E, Ns)
    P = spectrum(H, En, form)
    Pbar = bin_sum(P)
    if nbr is None:
        idx, val = peaks(Pbar, n_az, n_el, Ns, mask)
    else:
        idx, val = peaks_nbr(Pbar, nbr[0], nbr[1], Ns, mask)
    return dict(R=R, A=A, E=E, lam=lam, P=P, Pbar=Pbar, idx=idx, val=val)
