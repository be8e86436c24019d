"""FP64 CPU oracle of the GAP hot path (ctypes binding of gap_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and
by the cpu_baseline / reference legs of bench.py.  The product path (the
CUDA library and its binding) never imports, links or calls anything here.

Each function follows the paper's definitions literally; see the header of
gap_oracle.c for the equation each one restates and the readings taken
where the paper is silent.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gap_oracle.c")
# ORACLE_PLANT=k (k > 0) plants mistake k, for the tests that show the pins
# catch it: the mistakes in _PY_PLANTS switch on a line marked "planted k" in
# this module, the others load a build of gap_oracle.c compiled with that
# mistake; unset or 0: the oracle as written.
_PLANT = int(os.environ.get("ORACLE_PLANT", "0") or 0)
_PY_PLANTS = frozenset(range(16, 26)) | {32}
_C_PLANT = _PLANT if _PLANT and _PLANT not in _PY_PLANTS else 0
_LIB = os.path.join(_HERE, f"liboracle_plant{_C_PLANT}.so" if _C_PLANT else "liboracle.so")
_lib = None

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


class SoapParams(C.Structure):
    _fields_ = [("n_max", C.c_int), ("l_max", C.c_int), ("n_species", C.c_int), ("mix_K", C.c_int),
                ("rc", C.c_double), ("d", C.c_double), ("sigma", C.c_double), ("central_weight", C.c_double),
                ("mix_w", _dp), ("quad_n", C.c_int)]


class ModelParams(C.Structure):
    _fields_ = [("n_gp", C.c_int), ("m_offsets", _ip), ("sparse", _dp), ("alpha", _dp),
                ("delta", C.c_double), ("zeta", C.c_int), ("m2", C.c_int), ("x2", _dp), ("alpha2", _dp),
                ("delta2", C.c_double), ("theta2", C.c_double), ("rc2", C.c_double), ("d2", C.c_double)]


def build(force: bool = False) -> str:
    """Compile gap_oracle.c into liboracle.so (plain gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        plant = [f"-DORACLE_PLANT={_C_PLANT}"] if _C_PLANT else []
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", *plant, "-o", _LIB, _SRC, "-lm"])
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        L.orc_fcut.restype = C.c_double
        L.orc_fcut.argtypes = [C.c_double, C.c_double, C.c_double, _dp]
        L.orc_bessel_scaled.restype = C.c_double
        L.orc_bessel_scaled.argtypes = [C.c_int, C.c_double, _dp]
        L.orc_radial_basis.argtypes = [C.POINTER(SoapParams), C.c_double, _dp]
        L.orc_radial_integrals.argtypes = [C.POINTER(SoapParams), C.c_double, _dp, _dp]
        L.orc_ylm.argtypes = [C.c_int, _dp, _dp, _dp]
        L.orc_dim.argtypes = [C.POINTER(SoapParams)]
        L.orc_neighbours.restype = C.c_long
        L.orc_neighbours.argtypes = [C.c_int, _dp, _dp, _ip, C.c_double, C.c_int, C.c_long, _ip, _ip, _dp]
        L.orc_descriptor.argtypes = [C.POINTER(SoapParams), C.c_int, _dp, _ip, _dp, _ip, C.c_int, _ip, _dp, _dp, _dp]
        L.orc_predict.argtypes = [C.POINTER(SoapParams), C.POINTER(ModelParams), C.c_int, _dp, _ip, _dp, _ip,
                                  _dp, _dp, _dp, _dp]
        L.orc_predict_sampled.argtypes = [C.POINTER(SoapParams), C.POINTER(ModelParams), C.c_int, _dp, _ip, _dp,
                                          _ip, C.c_int, _ip, _dp, _dp]
        L.orc_knm.argtypes = [C.POINTER(SoapParams), C.POINTER(ModelParams), C.c_int, _dp, _ip, _dp, _ip, _dp]
        L.orc_kmm.argtypes = [C.POINTER(ModelParams), C.c_int, C.c_int, _dp]
        L.orc_solve_normal.argtypes = [C.c_long, C.c_int, _dp, _dp, _dp, _dp, C.c_double, _dp]
        L.orc_solve_qr.argtypes = [C.c_long, C.c_int, _dp, _dp, _dp, _dp, C.c_double, _dp]
        L.orc_num_threads.restype = C.c_int
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(_dp) if a is not None else None


def _i(a):
    return a.ctypes.data_as(_ip) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


class Soap:
    """SOAP hyperparameters (the `soap` keywords of the Appendix)."""

    def __init__(self, n_max, l_max, rc, sigma, d=1.0, central_weight=1.0, n_species=1, mix_K=0, mix_w=None,
                 quad_n=0):
        self.mix_w = None if mix_w is None else _f64(mix_w).reshape(-1)
        self.c = SoapParams(n_max, l_max, n_species, mix_K, rc, d, sigma, central_weight,
                            _d(self.mix_w), quad_n)

    @classmethod
    def from_spec(cls, spec, quad_n=0):
        return cls(spec.n_max, spec.l_max, spec.rc, spec.sigma, spec.d, spec.central_weight, spec.n_species,
                   spec.mix_K, spec.mix_w, quad_n)

    @property
    def dim(self) -> int:
        return lib().orc_dim(C.byref(self.c))


class Model:
    """Sparse GP per central species (+ optional two-body term)."""

    def __init__(self, sparse: list, alpha: list, delta: float, zeta: int, two_body=None):
        self.sparse = _f64(np.concatenate([np.asarray(s).reshape(-1, np.asarray(s).shape[-1]) for s in sparse]))
        self.alpha = _f64(np.concatenate([np.asarray(a).reshape(-1) for a in alpha]))
        self.offsets = _i32(np.concatenate([[0], np.cumsum([np.asarray(a).size for a in alpha])]))
        self.x2 = self.a2 = None
        m2, d2, t2, rc2, w2 = 0, 0.0, 1.0, 0.0, 1.0
        if two_body is not None:
            self.x2, self.a2 = _f64(two_body.x), _f64(two_body.alpha)
            m2, d2, t2, rc2, w2 = self.x2.size, two_body.delta, two_body.theta, two_body.rc, two_body.d
        self.c = ModelParams(len(alpha), _i(self.offsets), _d(self.sparse), _d(self.alpha), delta, int(zeta),
                             m2, _d(self.x2), _d(self.a2), d2, t2, rc2, w2)


def fcut(r, rc, d):
    df = C.c_double()
    f = lib().orc_fcut(r, rc, d, C.byref(df))
    return f, df.value


def bessel_scaled(l, x):
    """(e^-x i_l(x), e^-x i_l'(x))."""
    dv = C.c_double()
    v = lib().orc_bessel_scaled(l, x, C.byref(dv))
    return v, dv.value


def radial_basis(soap: Soap, r: float) -> np.ndarray:
    g = np.zeros(soap.c.n_max)
    lib().orc_radial_basis(C.byref(soap.c), r, _d(g))
    return g


def radial_integrals(soap: Soap, r: float):
    shape = (soap.c.n_max, soap.c.l_max + 1)
    I, dI = np.zeros(shape), np.zeros(shape)
    lib().orc_radial_integrals(C.byref(soap.c), r, _d(I), _d(dI))
    return I, dI


def ylm(L: int, u) -> tuple[np.ndarray, np.ndarray]:
    u = _f64(u)
    Y = np.zeros((L + 1) ** 2)
    dY = np.zeros(((L + 1) ** 2, 3))
    lib().orc_ylm(L, _d(u), _d(Y), _d(dY))
    return Y, dY


def neighbours(pos, cell, pbc, rc, i, cap=4096):
    pos, cell, pbc = _f64(pos), _f64(cell), _i32(pbc)
    j = np.zeros(cap, np.int32)
    sh = np.zeros((cap, 3), np.int32)
    v = np.zeros((cap, 3))
    m = lib().orc_neighbours(pos.shape[0], _d(pos), _d(cell), _i(pbc), rc, i, cap, _i(j), _i(sh), _d(v))
    if m > cap:
        return neighbours(pos, cell, pbc, rc, i, cap=int(m))
    return j[:m], sh[:m], v[:m]


def descriptor(soap: Soap, s, sel=None, with_coef=False):
    """Normalised power spectra p_hat [n_sel][D] and norms |p| of one structure."""
    pos, spec, cell, pbc = _f64(s.pos), _i32(s.species), _f64(s.cell), _i32(s.pbc)
    seli = None if sel is None else _i32(sel)
    ns = pos.shape[0] if sel is None else seli.size
    D = soap.dim
    ph = np.zeros((ns, D))
    pn = np.zeros(ns)
    G = soap.c.mix_K if soap.c.mix_K > 0 else 1
    Nc = soap.c.n_max if soap.c.mix_K > 0 else soap.c.n_max * soap.c.n_species
    coef = np.zeros((ns, G, Nc, (soap.c.l_max + 1) ** 2)) if with_coef else None
    lib().orc_descriptor(C.byref(soap.c), pos.shape[0], _d(pos), _i(spec), _d(cell), _i(pbc), ns, _i(seli),
                         _d(ph), _d(pn), _d(coef))
    return (ph, pn, coef) if with_coef else (ph, pn)


def predict(soap: Soap, model: Model, s):
    """(E, local energies [n], forces [n][3], virial [3][3]) of one structure."""
    pos, spec, cell, pbc = _f64(s.pos), _i32(s.species), _f64(s.cell), _i32(s.pbc)
    n = pos.shape[0]
    E = np.zeros(1)
    le = np.zeros(n)
    F = np.zeros((n, 3))
    V = np.zeros((3, 3))
    lib().orc_predict(C.byref(soap.c), C.byref(model.c), n, _d(pos), _i(spec), _d(cell), _i(pbc), _d(E), _d(le),
                      _d(F), _d(V))
    return float(E[0]), le, F, V


def predict_sampled(soap: Soap, model: Model, s, sel):
    """(local energies, forces) of the selected atoms of one structure."""
    pos, spec, cell, pbc = _f64(s.pos), _i32(s.species), _f64(s.cell), _i32(s.pbc)
    sel = _i32(sel)
    le = np.zeros(sel.size)
    F = np.zeros((sel.size, 3))
    lib().orc_predict_sampled(C.byref(soap.c), C.byref(model.c), pos.shape[0], _d(pos), _i(spec), _d(cell),
                              _i(pbc), sel.size, _i(sel), _d(le), _d(F))
    return le, F


def knm(soap: Soap, model: Model, s) -> np.ndarray:
    """K_NM rows [1 + 3n][M_total] of one structure: energy row, then (atom, xyz)."""
    pos, spec, cell, pbc = _f64(s.pos), _i32(s.species), _f64(s.cell), _i32(s.pbc)
    n = pos.shape[0]
    rows = np.zeros((1 + 3 * n, int(model.offsets[-1])))
    lib().orc_knm(C.byref(soap.c), C.byref(model.c), n, _d(pos), _i(spec), _d(cell), _i(pbc), _d(rows))
    return rows


def kmm(model: Model, D: int, s: int = 0) -> np.ndarray:
    M = int(model.offsets[s + 1] - model.offsets[s])
    out = np.zeros((M, M))
    lib().orc_kmm(C.byref(model.c), D, s, _d(out))
    return out


def solve_normal(K, y, sigma, Kmm, jitter):
    K, y, sigma, Kmm = _f64(K), _f64(y), _f64(sigma), _f64(Kmm)
    c = np.zeros(K.shape[1])
    st = lib().orc_solve_normal(K.shape[0], K.shape[1], _d(K), _d(y), _d(sigma), _d(Kmm), jitter, _d(c))
    if st:
        raise np.linalg.LinAlgError("K_MM + K^T S^-1 K is not positive definite")
    return c


def solve_qr(K, y, sigma, Kmm, jitter):
    K, y, sigma, Kmm = _f64(K), _f64(y), _f64(sigma), _f64(Kmm)
    c = np.zeros(K.shape[1])
    st = lib().orc_solve_qr(K.shape[0], K.shape[1], _d(K), _d(y), _d(sigma), _d(Kmm), jitter, _d(c))
    if st:
        raise np.linalg.LinAlgError("K_MM + jitter is not positive definite")
    return c


def num_threads() -> int:
    return lib().orc_num_threads()


def kernel_rows(soap: Soap, model: Model, s):
    """k_x [n][M_total] of every atom of structure s: delta^2 (p_hat_i . x_m)^zeta
    (Eqs. 2, 13) for the sparse points of the atom's own GP (its species),
    0 for the other GPs' columns; and k(x_i, x_i) [n]."""
    ph, _ = descriptor(soap, s)
    d2, z = model.c.delta ** 2, model.c.zeta
    k = np.zeros((ph.shape[0], int(model.offsets[-1])))
    for i in range(ph.shape[0]):
        g = int(s.species[i])
        a, b = int(model.offsets[g]), int(model.offsets[g + 1])
        k[i, a:b] = d2 * (model.sparse[a:b] @ ph[i]) ** z
    kxx = d2 * np.einsum("ij,ij->i", ph, ph) ** z
    return k, kxx


def predict_variance(soap: Soap, model: Model, s, knm_rows, sigma_rows, jitter):
    """Predictive variance of each local energy of structure s under the
    sparse GP whose coefficients Eq. 4 gives (the posterior of the projected
    process, with the jitter of Sec. 2 on K_MM):
        var(x) = k(x, x) - k_x^T Kt^-1 k_x + k_x^T (A^T A)^-1 k_x,
    Kt = K_MM + jitter I (block diagonal over the GPs), A = [S^-1/2 K_NM ; U]
    with Kt = U^T U (Eq. 5), S = diag(sigma_rows^2).  With A = QR (Eqs. 8-9),
    (A^T A)^-1 = R^-1 R^-T.  Steps: Cholesky of Kt, Householder QR of A
    (LAPACK, R only), two triangular solves per atom."""
    import scipy.linalg as sl
    D = soap.dim
    Mt = int(model.offsets[-1])
    Kt = np.zeros((Mt, Mt))
    for g in range(model.c.n_gp):
        a, b = int(model.offsets[g]), int(model.offsets[g + 1])
        Kt[a:b, a:b] = kmm(model, D, g)
    Kt += jitter * np.eye(Mt)
    U = sl.cholesky(Kt, lower=False)
    knm_rows = _f64(knm_rows).reshape(-1, Mt)
    A = np.vstack([knm_rows if _PLANT == 17 else knm_rows / _f64(sigma_rows)[:, None], U])  # planted 17: no S^-1/2
    R = sl.qr(A, mode="r")[0][:Mt]
    k, kxx = kernel_rows(soap, model, s)
    var = np.empty(k.shape[0])
    for i in range(k.shape[0]):
        v = sl.solve_triangular(U, k[i], trans="T")
        w = sl.solve_triangular(R, k[i], trans="T")
        var[i] = kxx[i] - v @ v + (-(w @ w) if _PLANT == 16 else w @ w)  # planted 16: sign
    return var


def cur_select(X, m, k=0, dup_tol=1e-10, rel_tol=1e-4):
    """'cur_points' sparse-point selection (Sec. 3.2.2; the CUR decomposition
    of Mahoney and Drineas, PNAS 106, 697 (2009), applied to the rows of the
    descriptor matrix X [n][D]): rank-k leverage scores
        pi_i = (1/k) sum_{xi < k} U_{i xi}^2,   X = U S V^T (thin SVD),
    then, deterministically, the rows with the m largest scores (equal scores:
    lower index first), skipping a row that duplicates an already chosen row
    within dup_tol in the max norm (duplicates are considered once, Sec.
    3.2.2).  k = 0 takes the numerical rank at singular values >= rel_tol
    times the largest, capped by m.  Returns (chosen indices in selection
    order, pi, k)."""
    X = _f64(X)
    n = X.shape[0]
    U, s, _ = np.linalg.svd(X, full_matrices=False)
    if k == 0:
        k = max(1, min(m, int((s >= rel_tol * s[0]).sum())))
    pi = (U[:, :k] ** 2).sum(axis=1) / (1 if _PLANT == 18 else k)  # planted 18: no 1/k
    order = np.lexsort((np.arange(n), pi if _PLANT == 20 else -pi))  # planted 20: smallest first
    chosen = []
    for i in order:
        if len(chosen) == m:
            break
        if _PLANT != 19 and any(np.abs(X[i] - X[j]).max() <= dup_tol for j in chosen):  # planted 19
            continue
        chosen.append(int(i))
    return np.array(chosen, dtype=np.int64), pi, k


def _ordered_power_spectrum(c, N, S, L):
    """P[a][b][l] = sum_m c_{a,lm} c_{b,lm} over all ordered channel pairs
    (a = species * N + n), Eq. 22 before any symmetric storage."""
    Nc = S * N
    P = np.zeros((Nc, Nc, L + 1))
    for l in range(L + 1):
        blk = c[:, l * l:(l + 1) * (l + 1)]
        P[:, :, l] = blk @ blk.T
    return P


def compressed_descriptor(soap: Soap, s, comp: dict):
    """Compressed, renormalised SOAP descriptors [n][D~] of structure s (Sec.
    3.3.3, and the compression recipes of soap_turbo, Sec. 3.3.4), from the
    expansion coefficients of the full multi-species descriptor (Eq. 23):
      'sketch'         p^k_l = (sum_{alpha n} w^k_{alpha n} c^alpha_{nl}) . (sum_{beta n'} u^k_{beta n'} c^beta_{n'l})
      'decomposition'  the same with u = w (sym_mix = T)
      'nu'             sums of p^{alpha beta}_{n n' l} over beta (nu_S = 1) or
                       alpha and beta (nu_S = 0), over n' (nu_R = 1) or n and
                       n' (nu_R = 0); output order (alpha, beta, n, n', l)
                       with the summed indices dropped
      'trivial'        the entries p_{n n' l} whose first radial index is the
                       first radial function of a species block, all n', l;
                       order (alpha, n', l) with n' over all channels
      'matrix'         P p for a user matrix P [D~][D] acting on the
                       uncompressed power spectrum p (this module's storage)
    then p~ / |p~| ("the descriptor is renormalized after compression")."""
    if soap.c.mix_K > 0:
        raise ValueError("compression acts on the fully coupled descriptor (mix_K = 0)")
    N, L, S = soap.c.n_max, soap.c.l_max, soap.c.n_species
    ph, pn, coef = descriptor(soap, s, with_coef=True)
    rec = comp["recipe"]
    out = []
    for i in range(ph.shape[0]):
        c = coef[i, 0]  # [S N][(L+1)^2]
        if rec in ("sketch", "decomposition"):
            w = np.asarray(comp["w"], dtype=np.float64)
            u = w if rec == "decomposition" or _PLANT == 21 else np.asarray(comp["u"], dtype=np.float64)  # planted 21
            cw, cu = w @ c, u @ c  # mixed channels [K][(L+1)^2]
            v = np.array([[cw[k, l * l:(l + 1) ** 2] @ cu[k, l * l:(l + 1) ** 2] for l in range(L + 1)]
                          for k in range(w.shape[0])]).ravel()
        elif rec == "nu":
            P = _ordered_power_spectrum(c, N, S, L).reshape(S, N, S, N, L + 1)  # [alpha][n][beta][n'][l]
            P = P.transpose(0, 2, 1, 3, 4)  # [alpha][beta][n][n'][l]
            nS, nR = comp["nu_S"], comp["nu_R"]
            if nS <= 1:
                P = P.sum(axis=0 if _PLANT == 22 and nS == 1 else 1, keepdims=True)  # planted 22: over alpha
            if nS == 0:
                P = P.sum(axis=0, keepdims=True)
            if nR <= 1:
                P = P.sum(axis=2 if _PLANT == 25 and nR == 1 else 3, keepdims=True)  # planted 25: over n
            if nR == 0:
                P = P.sum(axis=2, keepdims=True)
            v = P.ravel()
        elif rec == "trivial":
            P = _ordered_power_spectrum(c, N, S, L)
            v = np.stack([P[alpha if _PLANT == 23 else alpha * N] for alpha in range(S)]).ravel()  # planted 23
        elif rec == "matrix":
            v = np.asarray(comp["P"], dtype=np.float64) @ (ph[i] * pn[i])
        else:
            raise ValueError(rec)
        out.append(v if _PLANT == 24 else v / np.linalg.norm(v))  # planted 24: not renormalised
    return np.array(out)


def compressed_local_energies(soap: Soap, comp: dict, model: Model, s):
    """eps_i = delta^2 sum_m alpha_m (p~_i . x_m)^zeta (Eqs. 2, 13) on the
    compressed descriptors, sparse points x_m of the atom's own GP."""
    ph = compressed_descriptor(soap, s, comp)
    d2, z = model.c.delta ** 2, model.c.zeta
    eps = np.zeros(ph.shape[0])
    for i in range(ph.shape[0]):
        g = int(s.species[i])
        a, b = int(model.offsets[g]), int(model.offsets[g + 1])
        eps[i] = d2 * (model.alpha[a:b] * (model.sparse[a:b] @ ph[i]) ** (z + (_PLANT == 32))).sum()  # planted 32
    return eps
