"""Plant one plausible mistake at a time in a copy of the oracle (on the CPU)
and check that at least one pin catches it: the pins are not vacuous."""

import types

import numpy as np
import pytest

import oracle.gsvd_music as O
from oracle_pins import ALL_PINS


def _mutant(**overrides):
    ns = types.SimpleNamespace(**{k: getattr(O, k) for k in dir(O) if not k.startswith("__")})
    for k, v in overrides.items():
        setattr(ns, k, v)
    # localize_block must route through the mutated pieces
    def localize_block(X, K, H, Ns, n_az, n_el, form="abs"):
        R = ns.correlation(X)
        A, E, lam, _ = ns.gsvd(K, R)
        P = ns.spectrum(H, ns.noise_subspace(E, Ns), form)
        Pbar = ns.bin_sum(P)
        idx, val = ns.peaks(Pbar, n_az, n_el, Ns)
        return dict(R=R, A=A, E=E, lam=lam, P=P, Pbar=Pbar, idx=idx, val=val)
    ns.localize_block = localize_block
    return ns


def _no_conj_corr(X):
    X = np.asarray(X, complex)
    return np.einsum("tbi,tbj->bij", X, X) / X.shape[0]


def _no_scale_corr(X):
    X = np.asarray(X, complex)
    return np.einsum("tbi,tbj->bij", X, np.conj(X))


def _transposed_corr(X):
    X = np.asarray(X, complex)
    return np.einsum("tbi,tbj->bji", X, np.conj(X)) / X.shape[0]


def _right_whiten(K, R):
    return np.matmul(R, np.linalg.inv(K))


def _k_times_r(K, R):
    return np.matmul(K, R)


def _gsvd_right_vectors(K, R):
    A = O.whiten(K, R)
    U, s, Vh = np.linalg.svd(A)
    return A, np.conj(np.swapaxes(Vh, -1, -2)), s, U


def _gsvd_ascending(K, R):
    A = O.whiten(K, R)
    U, s, Vh = np.linalg.svd(A)
    return A, U[..., ::-1], s[..., ::-1], np.conj(np.swapaxes(Vh, -1, -2))[..., ::-1]


def _gsvd_of_r(K, R):
    return O.gsvd(np.broadcast_to(np.eye(R.shape[-1]), R.shape).astype(complex), R)


def _split_off_by_one(E, Ns):
    return E[..., :, Ns + 1:]


def _split_signal(E, Ns):
    return E[..., :, :Ns]


def _spectrum_swapped(H, En, form="abs"):
    return O.spectrum(H, En, "sq" if form == "abs" else "abs")


def _spectrum_no_conj(H, En, form="abs"):
    H = np.asarray(H, complex)
    Y = np.matmul(H, En)
    num = np.sum(np.abs(H) ** 2, axis=-1)
    den = np.sum(np.abs(Y), axis=-1) if form == "abs" else np.sum(np.abs(Y) ** 2, axis=-1)
    return num / np.maximum(den, 1e-300)


def _spectrum_no_num(H, En, form="abs"):
    P = O.spectrum(H, En, form)
    num = np.sum(np.abs(np.asarray(H)) ** 2, axis=-1)
    return P / num


def _bin_mean(P):
    return np.mean(P, axis=-2)


def _peaks_no_wrap(Pbar, n_az, n_el, Ns, mask=None):
    Pbar = np.asarray(Pbar, float)
    D = n_az * n_el
    cand = []
    for d in range(D):
        e, a = divmod(d, n_az)
        ok = True
        for ee in (e - 1, e, e + 1):
            for aa in (a - 1, a, a + 1):
                if not (0 <= ee < n_el and 0 <= aa < n_az):
                    continue
                n = ee * n_az + aa
                if n != d and not (Pbar[d] > Pbar[n] or (Pbar[d] == Pbar[n] and d < n)):
                    ok = False
        if ok and (mask is None or mask[d]):
            cand.append(d)
    cand.sort(key=lambda d: (-Pbar[d], d))
    idx = np.array((cand + [-1] * Ns)[:Ns])
    return idx, np.array([Pbar[d] if d >= 0 else 0.0 for d in idx])


def _peaks_ge(Pbar, n_az, n_el, Ns, mask=None):
    Pbar = np.asarray(Pbar, float)
    cand = []
    for d in range(n_az * n_el):
        e, a = divmod(d, n_az)
        ok = True
        for ee in (e - 1, e, e + 1):
            if not 0 <= ee < n_el:
                continue
            for aa in (a - 1, a, a + 1):
                n = ee * n_az + aa % n_az
                if n != d and Pbar[n] > Pbar[d]:
                    ok = False
        if ok and (mask is None or mask[d]):
            cand.append(d)
    cand.sort(key=lambda d: (-Pbar[d], d))
    idx = np.array((cand + [-1] * Ns)[:Ns])
    return idx, np.array([Pbar[d] if d >= 0 else 0.0 for d in idx])


def _sevd_ascending(R):
    lam, E = np.linalg.eigh(np.asarray(R, complex))
    return E, lam


def _gevd_wrong_side(K, R):
    # L^{-H} R L^{-1} instead of L^{-1} R L^{-H}
    L = np.linalg.cholesky(np.asarray(K, complex))
    Li = np.linalg.inv(L)
    LiH = np.conj(np.swapaxes(Li, -1, -2))
    lam, Y = np.linalg.eigh(np.matmul(np.matmul(LiH, np.asarray(R, complex)), Li))
    return np.matmul(LiH, Y)[..., ::-1], lam[..., ::-1]


def _gevd_no_backtransform(K, R):
    L = np.linalg.cholesky(np.asarray(K, complex))
    Li = np.linalg.inv(L)
    LiH = np.conj(np.swapaxes(Li, -1, -2))
    lam, Y = np.linalg.eigh(np.matmul(np.matmul(Li, np.asarray(R, complex)), LiH))
    return Y[..., ::-1], lam[..., ::-1]


def _margin_no_neighbours(Pbar, n_az, n_el, Ns, mask=None):
    Pbar = np.asarray(Pbar, dtype=np.float64)
    idx, _ = O.peaks(Pbar, n_az, n_el, Ns, mask)
    sel = [int(d) for d in idx if d >= 0]
    cand = _in(np.nonzero(O.is_peak(Pbar, n_az, n_el))[0], mask)
    rest = [Pbar[d] for d in cand if d not in sel]
    low = Pbar[sel[-1]]
    return float((low - max(rest)) / abs(low)) if rest else float("inf")


def _gap_absolute(lam, Ns):
    ln = np.asarray(lam, dtype=np.float64)[..., Ns:]
    if ln.shape[-1] < 2:
        return np.full(ln.shape[:-1], np.inf)
    return np.min(ln[..., :-1] - ln[..., 1:], axis=-1)


def _gap_from_signal(lam, Ns):
    return O.noise_gap(lam, Ns - 1)


def _peaks_nbr_variant(ge=False, drop_last=False, count_self=False):
    def peaks_nbr(Pbar, ptr, nbr, Ns, mask=None):
        Pbar = np.asarray(Pbar, dtype=np.float64)
        pk = []
        for d in range(Pbar.size):
            hi = ptr[d + 1] - (1 if drop_last and ptr[d + 1] > ptr[d] else 0)
            ok = True
            for n in nbr[ptr[d]:hi]:
                n = int(n)
                if n == d and not count_self:
                    continue
                beat = Pbar[d] >= Pbar[n] if ge else (Pbar[d] > Pbar[n] or
                                                      (Pbar[d] == Pbar[n] and d < n))
                ok = ok and beat
            if ok and (mask is None or mask[d]):
                pk.append(d)
        pk.sort(key=lambda d: (-Pbar[d], d))
        idx = np.full(Ns, -1, dtype=np.int64)
        val = np.zeros(Ns)
        for k, d in enumerate(pk[:Ns]):
            idx[k], val[k] = d, Pbar[d]
        return idx, val
    return peaks_nbr


def _margin_nbr_no_neighbours(Pbar, ptr, nbr, Ns, mask=None):
    Pbar = np.asarray(Pbar, dtype=np.float64)
    idx, _ = O.peaks_nbr(Pbar, ptr, nbr, Ns, mask)
    sel = [int(d) for d in idx if d >= 0]
    if not sel:
        return 0.0
    cand = _in(np.nonzero(O.is_peak_nbr(Pbar, ptr, nbr))[0], mask)
    rest = [Pbar[d] for d in cand if d not in sel]
    low = Pbar[sel[-1]]
    return float((low - max(rest)) / abs(low)) if rest else float("inf")


def _in(cand, mask):
    return cand if mask is None else np.asarray([d for d in cand if mask[d]], dtype=np.int64)


def _peaks_range_ignored(Pbar, n_az, n_el, Ns, mask=None):
    return O.peaks(Pbar, n_az, n_el, Ns)


def _peaks_range_restricts_neighbours(Pbar, n_az, n_el, Ns, mask=None):
    """Compares an in-range direction with its in-range neighbours only."""
    if mask is None:
        return O.peaks(Pbar, n_az, n_el, Ns)
    Pm = np.where(np.asarray(mask, bool), np.asarray(Pbar, float), -np.inf)
    idx, val = O.peaks(Pm, n_az, n_el, Ns, mask)
    return idx, val


def _peaks_nbr_range_ignored(Pbar, ptr, nbr, Ns, mask=None):
    return O.peaks_nbr(Pbar, ptr, nbr, Ns)


MUTANTS = {
    "peaks_nbr_ties_not_broken": dict(peaks_nbr=_peaks_nbr_variant(ge=True)),
    "peaks_nbr_drops_last_neighbour": dict(peaks_nbr=_peaks_nbr_variant(drop_last=True)),
    "peaks_nbr_compares_with_itself": dict(peaks_nbr=_peaks_nbr_variant(count_self=True)),
    "peak_margin_nbr_no_neighbour_term": dict(peak_margin_nbr=_margin_nbr_no_neighbours),
    "sevd_ascending": dict(sevd=_sevd_ascending),
    "gevd_wrong_side": dict(gevd=_gevd_wrong_side),
    "gevd_no_backtransform": dict(gevd=_gevd_no_backtransform),
    "corr_no_conj": dict(correlation=_no_conj_corr),
    "corr_no_1_over_T": dict(correlation=_no_scale_corr),
    "corr_transposed": dict(correlation=_transposed_corr),
    "whiten_right_side": dict(whiten=_right_whiten),
    "whiten_k_times_r": dict(whiten=_k_times_r),
    "gsvd_right_vectors": dict(gsvd=_gsvd_right_vectors),
    "gsvd_ascending": dict(gsvd=_gsvd_ascending),
    "gsvd_ignores_k": dict(gsvd=_gsvd_of_r),
    "split_off_by_one": dict(noise_subspace=_split_off_by_one),
    "split_signal_space": dict(noise_subspace=_split_signal),
    "spectrum_forms_swapped": dict(spectrum=_spectrum_swapped),
    "spectrum_no_conj": dict(spectrum=_spectrum_no_conj),
    "spectrum_no_numerator": dict(spectrum=_spectrum_no_num),
    "bin_mean_not_sum": dict(bin_sum=_bin_mean),
    "peaks_no_wrap": dict(peaks=_peaks_no_wrap),
    "peaks_plateau_duplicates": dict(peaks=_peaks_ge),
    "peak_margin_always_zero": dict(peak_margin=lambda Pbar, n_az, n_el, Ns, mask=None: 0.0),
    "peaks_range_ignored": dict(peaks=_peaks_range_ignored),
    "peaks_range_restricts_neighbours": dict(peaks=_peaks_range_restricts_neighbours),
    "peaks_nbr_range_ignored": dict(peaks_nbr=_peaks_nbr_range_ignored),
    "peak_margin_no_neighbour_term": dict(peak_margin=_margin_no_neighbours),
    "noise_gap_absolute": dict(noise_gap=_gap_absolute),
    "noise_gap_includes_last_signal_value": dict(noise_gap=_gap_from_signal),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name):
    ns = _mutant(**MUTANTS[name])
    # gsvd in the namespace must use the mutated whiten where it is mutated
    if "whiten" in MUTANTS[name]:
        w = MUTANTS[name]["whiten"]

        def gsvd(K, R):
            A = w(K, R)
            U, s, Vh = np.linalg.svd(A)
            return A, U, s, np.conj(np.swapaxes(Vh, -1, -2))
        ns.gsvd = gsvd
    caught = []
    for pin in ALL_PINS:
        try:
            pin(ns)
        except (AssertionError, ValueError, np.linalg.LinAlgError, IndexError):
            caught.append(pin.__name__)
    assert caught, f"no pin catches the planted mistake {name}"
