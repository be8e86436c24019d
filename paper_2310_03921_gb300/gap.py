"""Python binding of libgap (include/gap.h): argument marshalling only.

Every step of the hot path runs in the CUDA library; this module passes
pointers, sizes and the current stream.  It raises if libgap.so cannot be
loaded: there is no fallback implementation.

Arrays may be numpy (host) or torch CUDA tensors (device); the batch's
positions/species decide which, and outputs follow them.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgap.so")

GAP_FP64, GAP_BF16X3, GAP_FP32, GAP_BF16X6 = 0, 1, 2, 3
PRECISIONS = {"fp64": GAP_FP64, "bf16x3": GAP_BF16X3, "fp32": GAP_FP32, "bf16x6": GAP_BF16X6}
SOLVE_METHODS = {"householder": 0, "cholqr_tc": 1}
STATUS = {0: "GAP_OK", -1: "GAP_EINVAL", -2: "GAP_ENOMEM", -3: "GAP_ECUDA", -4: "GAP_ETIMEOUT", -5: "GAP_ENOTPD",
          -6: "GAP_EUNSUPPORTED", -7: "GAP_ECAPACITY"}

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)
_vp = C.c_void_p


class SoapParams(C.Structure):
    _fields_ = [("n_max", C.c_int), ("l_max", C.c_int), ("cutoff", C.c_double),
                ("cutoff_transition_width", C.c_double), ("atom_sigma", C.c_double),
                ("central_weight", C.c_double), ("n_species", C.c_int), ("mix_K", C.c_int), ("mix_w", _dp)]


class TwoBodyParams(C.Structure):
    _fields_ = [("n_sparse", C.c_int), ("cutoff", C.c_double), ("cutoff_transition_width", C.c_double),
                ("theta", C.c_double), ("delta", C.c_double), ("x", _dp), ("alpha", _dp)]


class CompressionStruct(C.Structure):
    _fields_ = [("recipe", C.c_int), ("K", C.c_int), ("w", _dp), ("u", _dp), ("nu_R", C.c_int), ("nu_S", C.c_int),
                ("d_out", C.c_int), ("P", _dp)]


COMPRESS = {"none": 0, "matrix": 1, "sketch": 2, "decomposition": 3, "nu": 4, "trivial": 5}


class BatchStruct(C.Structure):
    _fields_ = [("n_atoms", C.c_int), ("n_configs", C.c_int), ("config_offsets", _ip), ("cell", _dp),
                ("pbc", _ip), ("pos", _vp), ("species", _vp), ("device", C.c_int)]


class GapError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


_lib = None


def lib():
    """The loaded libgap.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libgap.so is missing at {LIB_PATH}; run paper_2310_03921_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        L.gap_last_error.restype = C.c_char_p
        L.gap_profile_stage_name.restype = C.c_char_p
        L.gap_profile_stage_name.argtypes = [C.c_int]
        L.gap_profile_stages.restype = C.c_int
        L.gap_launch_count.restype = C.c_long
        L.gap_tile_tuning_count.restype = C.c_int
        L.gap_step_graph_kernels.restype = C.c_long
        L.gap_step_graph_kernels.argtypes = [_vp]
        sig = {
            "gap_soap_create": [C.POINTER(SoapParams), C.POINTER(_vp)],
            "gap_soap_destroy": [_vp],
            "gap_soap_dim": [_vp, _ip],
            "gap_soap_cutoff": [_vp, _dp],
            "gap_soap_radial_table": [_vp, _ip, _dp],
            "gap_soap_set_compression": [_vp, C.POINTER(CompressionStruct)],
            "gap_descriptor_sizes": [_vp, C.POINTER(BatchStruct), C.POINTER(C.c_long), C.POINTER(C.c_long), _vp],
            "gap_descriptor": [_vp, C.POINTER(BatchStruct), C.c_int, _vp, _vp],
            "gap_model_create": [_vp, C.c_int, _ip, C.POINTER(_dp), C.POINTER(_dp), C.c_double, C.c_double,
                                 C.POINTER(TwoBodyParams), C.POINTER(_vp)],
            "gap_model_destroy": [_vp],
            "gap_step_graph_create": [_vp, C.POINTER(BatchStruct), C.c_int, C.c_double, _vp, _vp, _vp, _vp, _vp,
                                      C.POINTER(_vp)],
            "gap_step_graph_launch": [_vp, _vp],
            "gap_step_graph_status": [_vp, _vp],
            "gap_step_graph_destroy": [_vp],
            "gap_model_columns": [_vp, _ip],
            "gap_predict": [_vp, C.POINTER(BatchStruct), C.c_int, _vp, _vp, _vp, _vp, _vp],
            "gap_assemble_knm": [_vp, C.POINTER(BatchStruct), C.c_int, _vp, _vp],
            "gap_test_bf16_gemm": [C.c_int, C.c_int, C.c_int, C.c_int, _dp, _dp, _dp],
            "gap_gp_energy_noalloc": [_vp, C.c_int, C.c_int, _vp, _vp, _vp, _vp],
            "gap_solve": [_vp, C.c_long, _vp, _vp, _vp, C.c_double, C.c_int, _vp, C.c_int, _vp],
            "gap_fit": [_vp, _vp, C.c_int, _vp, _vp, C.c_double, C.c_int, _vp, C.c_int, _vp],
            "gap_test_f64_gemm": [C.c_int, C.c_int, C.c_int, _dp, _dp, C.c_int, _dp],
            "gap_test_f64_gram": [C.c_long, C.c_int, _dp, _dp],
            "gap_test_chol_inv": [C.c_int, _dp, _dp, _dp],
            "gap_test_product_crossover": [C.c_int, _dp, C.POINTER(C.c_float), _ip, C.POINTER(C.c_long)],
            "gap_test_congruence": [C.c_long, C.c_int, _dp, _dp, _dp, _dp, _dp, _dp, _dp],
            "gap_test_fma_peak": [C.c_int, _dp],
            "gap_test_tc_timeout": [C.c_ulonglong, _ip],
            "gap_test_fail_alloc": [C.c_long],
            "gap_test_tc_force_variant": [C.c_int],
            "gap_test_fp64_recip": [C.c_int, _dp, _dp],
            "gap_model_set_alpha": [_vp, _vp, C.c_int, _vp],
            "gap_model_set_posterior": [_vp, C.c_long, _vp, _vp, C.c_double, C.c_int, _vp],
            "gap_predict_variance": [_vp, C.POINTER(BatchStruct), _vp, _vp],
            "gap_cur_select": [_vp, C.c_long, C.c_int, C.c_int, C.c_int, C.c_double, C.c_int, _vp, _ip, _vp, _ip,
                               _vp],
            "gap_profile_enable": [C.c_int],
            "gap_profile_reset": [],
            "gap_profile_read": [_dp, _ip],
            "gap_tile_tuning_entry": [C.c_int, _ip, C.POINTER(C.c_float)],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.gap_test_bf16_gemm.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_float),
                                         C.POINTER(C.c_float), C.POINTER(C.c_float)]
        _lib = L
    return _lib


def _check(status: int):
    if status != 0:
        raise GapError(status, lib().gap_last_error().decode())


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _on_device(x) -> bool:
    """True for a CUDA torch tensor: its memory is passed as device memory.
    A torch tensor in host memory is passed as a host array."""
    return _is_torch(x) and bool(x.is_cuda)


def _host(x, dtype):
    """A contiguous numpy array of a host array or a CPU torch tensor."""
    if _is_torch(x):
        x = x.detach().cpu().numpy()
    return np.ascontiguousarray(x, dtype=dtype)


def _device_like(x, like, dtype="float64"):
    """x as a contiguous CUDA tensor on the device of `like` (copied there if
    it is a host array or a CPU tensor)."""
    import torch
    dt = getattr(torch, dtype)
    if _on_device(x) and x.device == like.device and x.dtype == dt:
        return x.contiguous()
    return torch.as_tensor(_host(x, dtype) if not _is_torch(x) else x, dtype=dt, device=like.device).contiguous()


def _ptr(x):
    if x is None:
        return None
    if _is_torch(x):
        return C.c_void_p(x.data_ptr())
    return x.ctypes.data_as(C.c_void_p)


def _stream(stream):
    if stream is not None:
        return C.c_void_p(stream)
    import torch
    if torch.cuda.is_available() and torch.cuda.is_initialized():
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return None


class Batch:
    """Configurations for one call.  Metadata is host numpy; positions/species
    are numpy (host) or torch CUDA tensors (device)."""

    def __init__(self, pos, species, cell, pbc, config_offsets):
        self.cell = np.ascontiguousarray(cell, dtype=np.float64).reshape(-1, 3, 3)
        self.pbc = np.ascontiguousarray(pbc, dtype=np.int32).reshape(-1, 3)
        self.offsets = np.ascontiguousarray(config_offsets, dtype=np.int32)
        self.device = _on_device(pos)
        if self.device:
            if str(pos.dtype) != "torch.float64":
                raise TypeError(f"device positions must be float64, not {pos.dtype}")
            if not (_on_device(species) and str(species.dtype) == "torch.int32" and species.device == pos.device):
                raise TypeError("with device positions, species must be an int32 tensor on the same device")
            self.pos = pos.contiguous()
            self.species = species.contiguous()
        else:
            self.pos = _host(pos, np.float64).reshape(-1, 3)
            self.species = _host(species, np.int32)
        self.n_atoms = int(self.pos.shape[0])
        self.n_configs = int(self.cell.shape[0])
        self.c = BatchStruct(self.n_atoms, self.n_configs, self.offsets.ctypes.data_as(_ip),
                             self.cell.ctypes.data_as(_dp), self.pbc.ctypes.data_as(_ip), _ptr(self.pos),
                             _ptr(self.species), 1 if self.device else 0)

    @classmethod
    def from_synth(cls, b, device=None):
        """From a synth.Batch (host); device='cuda' copies positions/species to the GPU."""
        if device is None:
            return cls(b.pos, b.species, b.cell, b.pbc, b.config_offsets)
        import torch
        return cls(torch.as_tensor(b.pos, dtype=torch.float64, device=device),
                   torch.as_tensor(b.species, dtype=torch.int32, device=device), b.cell, b.pbc, b.config_offsets)

    def empty(self, *shape):
        if self.device:
            import torch
            return torch.empty(*shape, dtype=torch.float64, device=self.pos.device)
        return np.empty(shape, dtype=np.float64)


class Soap:
    """gap_soap: the SOAP descriptor object (initialise/cutoff/sizes/calc/finalise)."""

    def __init__(self, n_max, l_max, cutoff, atom_sigma, cutoff_transition_width=1.0, central_weight=1.0,
                 n_species=1, mix_K=0, mix_w=None):
        self._mix = None if mix_w is None else np.ascontiguousarray(mix_w, dtype=np.float64).reshape(-1)
        p = SoapParams(n_max, l_max, cutoff, cutoff_transition_width, atom_sigma, central_weight, n_species, mix_K,
                       self._mix.ctypes.data_as(_dp) if self._mix is not None else None)
        h = C.c_void_p()
        _check(lib().gap_soap_create(C.byref(p), C.byref(h)))
        self.h = h
        self.n_max, self.l_max, self.n_species = n_max, l_max, n_species

    @classmethod
    def from_spec(cls, s):
        return cls(s.n_max, s.l_max, s.rc, s.sigma, s.d, s.central_weight, s.n_species, s.mix_K, s.mix_w)

    def close(self):
        if getattr(self, "h", None):
            lib().gap_soap_destroy(self.h)
            self.h = None

    __del__ = close

    @property
    def dim(self) -> int:
        d = C.c_int()
        _check(lib().gap_soap_dim(self.h, C.byref(d)))
        return d.value

    @property
    def cutoff(self) -> float:
        r = C.c_double()
        _check(lib().gap_soap_cutoff(self.h, C.byref(r)))
        return r.value

    def radial_table(self) -> np.ndarray:
        k = C.c_int()
        _check(lib().gap_soap_radial_table(self.h, C.byref(k), None))
        out = np.zeros((k.value, self.n_max, self.l_max + 1, 2))
        _check(lib().gap_soap_radial_table(self.h, C.byref(k), out.ctypes.data_as(_dp)))
        return out

    def set_compression(self, recipe="none", w=None, u=None, nu_S=2, nu_R=2, P=None):
        """Compress the descriptor (gap_soap_set_compression): recipe 'sketch'
        (w, u [K][Nc]), 'decomposition' (w), 'nu' (nu_S, nu_R), 'trivial',
        'matrix' (P [d_out][D]) or 'none'."""
        keep = []

        def arr(a):
            if a is None:
                return None, 0
            a = np.ascontiguousarray(a, dtype=np.float64)
            keep.append(a)
            return a.ctypes.data_as(_dp), a.shape[0]

        wp, K = arr(w)
        up, _ = arr(u)
        Pp, d_out = arr(P)
        c = CompressionStruct(COMPRESS[recipe], K, wp, up, int(nu_R), int(nu_S), d_out, Pp)
        _check(lib().gap_soap_set_compression(self.h, C.byref(c)))

    def descriptor_sizes(self, batch: Batch, stream=None):
        nd, npairs = C.c_long(), C.c_long()
        _check(lib().gap_descriptor_sizes(self.h, C.byref(batch.c), C.byref(nd), C.byref(npairs), _stream(stream)))
        return nd.value, npairs.value

    def descriptor(self, batch: Batch, precision="fp64", stream=None):
        out = batch.empty(batch.n_atoms, self.dim)
        _check(lib().gap_descriptor(self.h, C.byref(batch.c), PRECISIONS[precision], _ptr(out), _stream(stream)))
        return out


class Model:
    """gap_model: one dot-product sparse GP per central species (+ two-body term)."""

    def __init__(self, soap: Soap, sparse, alpha, delta, zeta, two_body=None):
        self.soap = soap
        D = soap.dim
        self._sp = [np.ascontiguousarray(np.asarray(s, dtype=np.float64).reshape(-1, D)) for s in sparse]
        self._al = [np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1)) for a in alpha]
        G = len(self._sp)
        M = (C.c_int * G)(*[s.shape[0] for s in self._sp])
        sp = (_dp * G)(*[s.ctypes.data_as(_dp) for s in self._sp])
        al = (_dp * G)(*[a.ctypes.data_as(_dp) for a in self._al])
        tbp = None
        if two_body is not None:
            self._tbx = np.ascontiguousarray(two_body.x, dtype=np.float64)
            self._tba = np.ascontiguousarray(two_body.alpha, dtype=np.float64)
            tbp = TwoBodyParams(self._tbx.size, two_body.rc, two_body.d, two_body.theta, two_body.delta,
                                self._tbx.ctypes.data_as(_dp), self._tba.ctypes.data_as(_dp))
        h = C.c_void_p()
        _check(lib().gap_model_create(soap.h, G, M, sp, al, float(delta), float(zeta),
                                      C.byref(tbp) if tbp is not None else None, C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().gap_model_destroy(self.h)
            self.h = None

    __del__ = close

    @property
    def columns(self) -> int:
        m = C.c_int()
        _check(lib().gap_model_columns(self.h, C.byref(m)))
        return m.value

    def predict(self, batch: Batch, precision="bf16x3", local=True, forces=True, virial=True, stream=None):
        """Dict with energy [C], local_e [N], forces [N][3], virial [C][3][3]."""
        E = batch.empty(batch.n_configs)
        le = batch.empty(batch.n_atoms) if local else None
        F = batch.empty(batch.n_atoms, 3) if forces else None
        V = batch.empty(batch.n_configs, 3, 3) if virial else None
        _check(lib().gap_predict(self.h, C.byref(batch.c), PRECISIONS[precision], _ptr(E), _ptr(le), _ptr(F),
                                 _ptr(V), _stream(stream)))
        return {"energy": E, "local_e": le, "forces": F, "virial": V}

    def set_alpha(self, alpha, stream=None):
        """Replace the coefficients (all GPs, column order) from numpy or a CUDA tensor."""
        dev = _on_device(alpha)
        a = _device_like(alpha, alpha) if dev else _host(alpha, np.float64)
        _check(lib().gap_model_set_alpha(self.h, _ptr(a), 1 if dev else 0, _stream(stream)))

    def solve(self, knm, y, sigma, jitter=1e-8, method="cholqr_tc", stream=None):
        """Regularised least-squares coefficients [M_total] (arrays host numpy or
        device torch); method 'cholqr_tc' (shifted CholeskyQR3 with tensor-core
        FP64 products) or 'householder' (FP64 Householder QR)."""
        dev = _on_device(knm)
        if dev:
            import torch
            out = torch.empty(self.columns, dtype=torch.float64, device=knm.device)
            knm, y, sigma = _device_like(knm, knm), _device_like(y, knm), _device_like(sigma, knm)
        else:
            knm, y, sigma = _host(knm, np.float64), _host(y, np.float64), _host(sigma, np.float64)
            out = np.empty(self.columns, dtype=np.float64)
        _check(lib().gap_solve(self.h, int(knm.shape[0]), _ptr(knm), _ptr(y), _ptr(sigma), float(jitter),
                               SOLVE_METHODS[method], _ptr(out), 1 if dev else 0, _stream(stream)))
        return out

    def fit(self, batch: Batch, y, sigma, jitter=1e-8, method="cholqr_tc", precision="bf16x3", stream=None):
        """K_NM of the batch, the regularised least-squares solve and the new
        coefficients installed in the model, in one call (K_NM stays on the
        device).  y and sigma in K_NM row order, host numpy or device torch;
        returns the coefficients in the same memory."""
        dev = _on_device(y)
        if dev:
            import torch
            out = torch.empty(self.columns, dtype=torch.float64, device=y.device)
            y, sigma = _device_like(y, y), _device_like(sigma, y)
        else:
            y, sigma = _host(y, np.float64), _host(sigma, np.float64)
            out = np.empty(self.columns, dtype=np.float64)
        _check(lib().gap_fit(self.h, C.byref(batch.c), PRECISIONS[precision], _ptr(y), _ptr(sigma), float(jitter),
                             SOLVE_METHODS[method], _ptr(out), 1 if dev else 0, _stream(stream)))
        return out

    def set_posterior(self, knm, sigma, jitter=1e-8, stream=None):
        """Keep the posterior factors of the fit on training rows knm
        [rows][M_total] with per-row sigma (host numpy or device torch), for
        predict_variance."""
        dev = _on_device(knm)
        if dev:
            knm, sigma = _device_like(knm, knm), _device_like(sigma, knm)
        else:
            knm = _host(knm, np.float64).reshape(-1, self.columns)
            sigma = _host(sigma, np.float64)
        _check(lib().gap_model_set_posterior(self.h, int(knm.shape[0]), _ptr(knm), _ptr(sigma), float(jitter),
                                             1 if dev else 0, _stream(stream)))

    def predict_variance(self, batch: Batch, stream=None):
        """Predictive variance [N] of each atom's local energy (FP64)."""
        out = batch.empty(batch.n_atoms)
        _check(lib().gap_predict_variance(self.h, C.byref(batch.c), _ptr(out), _stream(stream)))
        return out

    def assemble_knm(self, batch: Batch, precision="bf16x3", stream=None):
        out = batch.empty(batch.n_configs + 3 * batch.n_atoms, self.columns)
        _check(lib().gap_assemble_knm(self.h, C.byref(batch.c), PRECISIONS[precision], _ptr(out), _stream(stream)))
        return out


class StepGraph:
    """gap_step_graph: one predict of a fixed batch layout (device positions
    and species, read at every launch) captured as a CUDA graph.  Move the
    atoms by writing batch.pos in place, then launch(); outputs land in the
    tensors of `outputs`.  status() synchronises and raises GAP_ECAPACITY when
    the last launch had more pairs than the capacity."""

    def __init__(self, model: Model, batch: Batch, precision="bf16x3", pair_capacity=1.2, local=False,
                 forces=True, virial=True, stream=None):
        if not batch.device:
            raise ValueError("a step graph needs device positions and species")
        self.model, self.batch = model, batch
        self.outputs = {"energy": batch.empty(batch.n_configs),
                        "local_e": batch.empty(batch.n_atoms) if local else None,
                        "forces": batch.empty(batch.n_atoms, 3) if forces else None,
                        "virial": batch.empty(batch.n_configs, 3, 3) if virial else None}
        o = self.outputs
        h = C.c_void_p()
        _check(lib().gap_step_graph_create(model.h, C.byref(batch.c), PRECISIONS[precision], float(pair_capacity),
                                           _ptr(o["energy"]), _ptr(o["local_e"]), _ptr(o["forces"]),
                                           _ptr(o["virial"]), _stream(stream), C.byref(h)))
        self.h = h

    def launch(self, stream=None):
        _check(lib().gap_step_graph_launch(self.h, _stream(stream)))

    def status(self, stream=None):
        _check(lib().gap_step_graph_status(self.h, _stream(stream)))

    @property
    def kernels(self) -> int:
        return int(lib().gap_step_graph_kernels(self.h))

    def close(self):
        if getattr(self, "h", None):
            lib().gap_step_graph_destroy(self.h)
            self.h = None

    __del__ = close


_ENERGY_FN = None


def _energy_function():
    """The torch.autograd.Function around gap_predict, built on first use so
    that importing this module does not import torch."""
    global _ENERGY_FN
    if _ENERGY_FN is not None:
        return _ENERGY_FN
    import torch
    from torch.autograd.function import once_differentiable

    class GapEnergy(torch.autograd.Function):
        """E(r) of Eq. 1 with dE/dr from the library's backward kernels (Eq. 3):
        forward runs gap_predict (energies only when no gradient is needed),
        backward scales the forces it returned by the upstream gradient."""

        @staticmethod
        def forward(ctx, pos, model, species, cell, pbc, config_offsets, precision):
            b = Batch(pos.detach(), species, cell, pbc, config_offsets)
            grad = ctx.needs_input_grad[0]
            out = model.predict(b, precision, local=False, forces=grad, virial=grad)
            if grad:
                counts = torch.as_tensor(np.diff(b.offsets), dtype=torch.long, device=pos.device)
                ctx.save_for_backward(out["forces"], counts)
                ctx.mark_non_differentiable(out["virial"])
                return out["energy"], out["virial"]
            return out["energy"], None

        @staticmethod
        @once_differentiable
        def backward(ctx, g_energy, g_virial):
            forces, counts = ctx.saved_tensors
            per_atom = torch.repeat_interleave(g_energy, counts, output_size=forces.shape[0])
            return -per_atom[:, None] * forces, None, None, None, None, None, None

    _ENERGY_FN = GapEnergy
    return GapEnergy


def energy(model: "Model", pos, species, cell, pbc, config_offsets, precision="bf16x3"):
    """Energies [C] (FP64) as a differentiable function of the positions
    `pos` (a CUDA float64 tensor [N][3]); the virial [C][3][3] comes back
    beside them (None when pos does not require a gradient).  Gradients with
    respect to pos are -F from gap_predict's backward kernels, scaled per
    configuration by the upstream gradient; second derivatives are not
    provided."""
    if not (_on_device(pos) and str(pos.dtype) == "torch.float64"):
        raise TypeError("energy() needs the positions as a CUDA float64 tensor")
    return _energy_function().apply(pos, model, species, cell, pbc, config_offsets, precision)


def cur_select(X, m: int, k: int = 0, dup_tol: float = 1e-10, stream=None):
    """'cur_points' selection among the rows of X [n][D] (host numpy or CUDA
    tensor): (chosen row indices in selection order, leverage scores, k used)."""
    dev = _on_device(X)
    n, D = X.shape
    if dev:
        import torch
        X = _device_like(X, X)
        sel = torch.empty(m, dtype=torch.int32, device=X.device)
        sc = torch.empty(n, dtype=torch.float64, device=X.device)
    else:
        X = _host(X, np.float64)
        sel = np.empty(m, dtype=np.int32)
        sc = np.empty(n, dtype=np.float64)
    cnt, ku = C.c_int(), C.c_int()
    _check(lib().gap_cur_select(_ptr(X), n, D, int(k), int(m), float(dup_tol), 1 if dev else 0, _ptr(sel),
                                C.byref(cnt), _ptr(sc), C.byref(ku), _stream(stream)))
    return sel[:cnt.value], sc, ku.value


def profile_enable(on: bool = True):
    _check(lib().gap_profile_enable(1 if on else 0))


def profile_reset():
    _check(lib().gap_profile_reset())


def profile_read() -> dict:
    """{stage: (total ms, intervals)} since the last reset."""
    n = lib().gap_profile_stages()
    ms = np.zeros(n)
    cnt = np.zeros(n, dtype=np.int32)
    _check(lib().gap_profile_read(ms.ctypes.data_as(_dp), cnt.ctypes.data_as(_ip)))
    return {lib().gap_profile_stage_name(k).decode(): (float(ms[k]), int(cnt[k])) for k in range(n)}


def launch_count() -> int:
    return int(lib().gap_launch_count())


EPILOGUES = {0: "store", 1: "kernel", 2: "qpow", 3: "knm"}


def tile_tuning() -> list:
    """The tile autotuner's choices, one dict per tuned shape class."""
    out = []
    for k in range(lib().gap_tile_tuning_count()):
        f = (C.c_int * 8)()
        ms = (C.c_float * 4)()
        _check(lib().gap_tile_tuning_entry(k, f, ms))
        out.append({"epilogue": EPILOGUES.get(f[0], f[0]), "planes": f[1], "K": f[2], "cols": f[3],
                    "rows_log2": f[4], "tile": [128, f[5]], "stages": f[6],
                    "ms_256x2_128x2_128x3_192x2w12": [round(float(x), 4) for x in ms]})
    return out


def test_bf16_gemm(A: np.ndarray, B: np.ndarray, nsplit: int = 2) -> np.ndarray:
    """C = A B^T through the tensor-core test hook (host float32 arrays)."""
    A = np.ascontiguousarray(A, dtype=np.float32)
    B = np.ascontiguousarray(B, dtype=np.float32)
    Cm = np.zeros((A.shape[0], B.shape[0]), dtype=np.float32)
    fp = C.POINTER(C.c_float)
    _check(lib().gap_test_bf16_gemm(nsplit, A.shape[0], B.shape[0], A.shape[1], A.ctypes.data_as(fp),
                                    B.ctypes.data_as(fp), Cm.ctypes.data_as(fp)))
    return Cm


def test_f64_gemm(A: np.ndarray, B: np.ndarray, b_lower: bool = False) -> np.ndarray:
    """C = A B^T through the modular FP64 tensor-core product (host float64)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    Cm = np.zeros((A.shape[0], B.shape[0]))
    _check(lib().gap_test_f64_gemm(A.shape[0], B.shape[0], A.shape[1], A.ctypes.data_as(_dp), B.ctypes.data_as(_dp),
                                   1 if b_lower else 0, Cm.ctypes.data_as(_dp)))
    return Cm


def test_f64_gram(Y: np.ndarray) -> np.ndarray:
    """G = Y^T Y through the symmetric modular FP64 tensor-core product."""
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    G = np.zeros((Y.shape[1], Y.shape[1]))
    _check(lib().gap_test_f64_gram(Y.shape[0], Y.shape[1], Y.ctypes.data_as(_dp), G.ctypes.data_as(_dp)))
    return G


def test_chol_inv(Gm: np.ndarray):
    """(R, X): upper Cholesky factor of an SPD matrix and its inverse, by the
    recursive tensor-core factorisation (host float64)."""
    n = Gm.shape[0]
    Gf = np.asfortranarray(Gm, dtype=np.float64)
    R = np.zeros((n, n), order="F")
    X = np.zeros((n, n), order="F")
    _check(lib().gap_test_chol_inv(n, Gf.ctypes.data_as(_dp), R.ctypes.data_as(_dp), X.ctypes.data_as(_dp)))
    return R, X


def test_congruence(Y: np.ndarray, b: np.ndarray, Kt, W: np.ndarray):
    """(G, c, Wt) of the exact congruence of the CholeskyQR solve:
    G = Wt^T (Y^T Y + Kt) Wt and c = Wt^T Y^T b, with Wt the W the modular
    representation holds (host float64)."""
    m, n = Y.shape
    Yc = np.ascontiguousarray(Y, dtype=np.float64)
    bc = np.ascontiguousarray(b, dtype=np.float64)
    Kf = None if Kt is None else np.asfortranarray(Kt, dtype=np.float64)
    Wf = np.asfortranarray(W, dtype=np.float64)
    G = np.zeros((n, n), order="F")
    c = np.zeros(n)
    Wt = np.zeros((n, n), order="F")
    _check(lib().gap_test_congruence(m, n, Yc.ctypes.data_as(_dp) if m else None,
                                     bc.ctypes.data_as(_dp) if m else None,
                                     None if Kf is None else Kf.ctypes.data_as(_dp), Wf.ctypes.data_as(_dp),
                                     G.ctypes.data_as(_dp), c.ctypes.data_as(_dp), Wt.ctypes.data_as(_dp)))
    return G, c, Wt


def product_crossover(Gm: np.ndarray):
    """The factorisation's block-product tuner: ({size: (fp64_ms, modular_ms)},
    threshold multiply-adds)."""
    n = Gm.shape[0]
    Gf = np.asfortranarray(Gm, dtype=np.float64)
    ms = (C.c_float * 16)()
    sizes, thr = C.c_int(), C.c_long()
    _check(lib().gap_test_product_crossover(n, Gf.ctypes.data_as(_dp), ms, C.byref(sizes), C.byref(thr)))
    return {32 << k: (ms[k], ms[8 + k]) for k in range(sizes.value)}, thr.value


def fma_peak_tflops(fp64: bool = False) -> float:
    """Measured FP32 (or FP64) FMA throughput of the current GPU, TFLOP/s."""
    t = C.c_double()
    _check(lib().gap_test_fma_peak(1 if fp64 else 0, C.byref(t)))
    return t.value


def test_tc_timeout(wait_ns: int = 20000):
    """(status, error bits) of the tensor-core GEMM's bounded-wait test."""
    code = C.c_int()
    st = lib().gap_test_tc_timeout(int(wait_ns), C.byref(code))
    return st, code.value


def test_fail_alloc(after: int):
    """Make the library's workspace allocations fail after `after` more (-1: off)."""
    _check(lib().gap_test_fail_alloc(int(after)))


def test_tc_force_variant(v: int):
    """Force the contractions' tile variant (0..3, the autotuner's order; -1: tuner)."""
    _check(lib().gap_test_tc_force_variant(int(v)))


def test_fp64_recip(x: np.ndarray) -> np.ndarray:
    """[n][4]: the factorisation's FP64 reciprocal and rsqrt, CUDA's 1/x and rsqrt."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros((x.size, 4))
    _check(lib().gap_test_fp64_recip(x.size, x.ctypes.data_as(_dp), out.ctypes.data_as(_dp)))
    return out


def exported_symbols() -> list[str]:
    """Names declared by include/gap.h and include/gap_testing.h."""
    import re
    names = []
    for h in ("gap.h", "gap_testing.h"):
        txt = open(os.path.join(_HERE, "..", "include", h)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names += re.findall(r"\b(gap_[a-z0-9_]+)\s*\(", txt)
    return sorted(set(names))
