"""Thin Python binding of libdwsolve (include/dwsolve.h).

Argument marshalling only: every function forwards to the C entry point of
the same name with raw pointers taken from torch tensors.  All arithmetic
runs in the CUDA library; if the library is missing this module raises
instead of computing anything itself.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdwsolve.so")

DW_OK, DW_EINVAL, DW_ENOMEM, DW_ECUDA, DW_ENOTCONV, DW_ILLCOND = 0, -1, -2, -3, 1, 2
DW_F64, DW_F32, DW_BF16, DW_F64X = 0, 1, 2, 3
DW_OP_FULL, DW_OP_SCHUR = 0, 1


class DwError(RuntimeError):
    def __init__(self, rc, msg):
        super().__init__(f"dwsolve error {rc}: {msg}")
        self.rc = rc


class DwParams(C.Structure):
    _fields_ = [("L", C.c_int * 4), ("m0", C.c_double), ("csw", C.c_double), ("antiperiodic", C.c_int),
                ("sap_bs", C.c_int * 4)]


class DflParams(C.Structure):
    _fields_ = [("bs", C.c_int * 4), ("Ns", C.c_int), ("n_inv", C.c_int), ("ncy", C.c_int), ("nmr", C.c_int),
                ("basis_prec", C.c_int), ("iter_prec", C.c_int), ("cond_max", C.c_double),
                ("net_weights", C.c_void_p), ("net_channels", C.c_int), ("net_k0", C.c_int),
                ("net_judge", C.c_double), ("boot_steps", C.c_int), ("boot_tol", C.c_double),
                ("boot_nmx", C.c_int)]


class DflInfo(C.Structure):
    _fields_ = [("seconds", C.c_double), ("seconds_little", C.c_double), ("max_block_cond", C.c_double),
                ("Nb", C.c_int), ("N", C.c_int), ("learned_used", C.c_int), ("rho_in", C.c_double),
                ("rho_out", C.c_double), ("boot_steps", C.c_int), ("boot_gcr_steps", C.c_int),
                ("little_loaded", C.c_int)]


class SolParams(C.Structure):
    _fields_ = [("tol", C.c_double), ("nkv", C.c_int), ("nmx", C.c_int), ("ncy", C.c_int), ("nmr", C.c_int),
                ("mixed", C.c_int), ("inner_rtol", C.c_double), ("little_tol_out", C.c_double),
                ("little_tol_in", C.c_double), ("little_tol_cap", C.c_double), ("little_nkv", C.c_int),
                ("little_maxit", C.c_int)]


class SolInfo(C.Structure):
    _fields_ = [("status", C.c_int), ("iterations", C.c_int), ("restarts", C.c_int),
                ("little_iterations", C.c_int), ("little_solves", C.c_int), ("relres", C.c_double),
                ("seconds", C.c_double), ("t_sap", C.c_double), ("t_dirac", C.c_double),
                ("t_project", C.c_double), ("t_little", C.c_double), ("t_orth", C.c_double),
                ("t_restart", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_P = C.c_void_p
_SIGNATURES = {
    "dw_last_error": (C.c_char_p, []),
    "dw_launch_count": (C.c_longlong, []),
    "dw_create": (C.c_int, [C.POINTER(DwParams), _P, C.POINTER(_P)]),
    "dw_destroy": (None, [_P]),
    "dw_release_workspace": (C.c_int, [_P]),
    "dw_field_bytes": (C.c_size_t, [_P, C.c_int]),
    "dw_volume": (C.c_longlong, [_P]),
    "dw_pack": (C.c_int, [_P, C.c_int, C.c_int, _P, _P, _P]),
    "dw_unpack": (C.c_int, [_P, C.c_int, C.c_int, _P, _P, _P]),
    "dw_apply": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, _P, _P, _P]),
    "dw_apply_schur_static": (C.c_int, [_P, C.c_int, _P, _P, _P]),
    "sap_precondition": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.c_int, _P, _P, _P]),
    "deflation_build": (C.c_int, [_P, C.POINTER(DflParams), _P, C.POINTER(_P), C.POINTER(DflInfo)]),
    "dfl_destroy": (None, [_P]),
    "dfl_dims": (C.c_int, [_P, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "dfl_retarget": (C.c_int, [_P, _P, C.POINTER(_P), C.POINTER(DflInfo)]),
    "dfl_save": (C.c_int, [_P, C.c_char_p]),
    "dfl_load": (C.c_int, [_P, C.c_char_p, C.POINTER(_P), C.POINTER(DflInfo)]),
    "dfl_restrict": (C.c_int, [_P, C.c_int, _P, _P, _P]),
    "dfl_prolong": (C.c_int, [_P, C.c_int, _P, _P, _P]),
    "dfl_basis_export": (C.c_int, [_P, _P, _P]),
    "little_apply": (C.c_int, [_P, _P, _P, _P]),
    "little_dirac_solve": (C.c_int, [_P, C.c_int, _P, _P, C.c_double, C.c_int, C.POINTER(C.c_int),
                                     C.POINTER(C.c_double), _P]),
    "little_dirac_solve_batch": (C.c_int, [_P, C.c_int, C.c_int, _P, _P, C.c_double, C.c_int, C.POINTER(C.c_int),
                                           C.POINTER(C.c_double), _P]),
    "gcr_solve": (C.c_int, [_P, _P, C.POINTER(SolParams), C.c_int, _P, _P, C.POINTER(SolInfo), _P]),
    "dw_autotune": (C.c_int, [_P, C.c_int, C.c_char_p, C.c_size_t]),
    "dfl_autotune": (C.c_int, [_P, C.c_char_p, C.c_size_t]),
    "cgnr_solve": (C.c_int, [_P, C.c_double, C.c_int, _P, _P, C.POINTER(C.c_int), C.POINTER(C.c_double), _P]),
    "lowmodes_solve": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.c_double, C.c_int, C.c_int, _P, _P,
                                 C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_int), _P]),
    "dfl_deficits": (C.c_int, [_P, C.c_int, _P, C.POINTER(C.c_double), _P]),
    "bicgstab_solve": (C.c_int, [_P, C.c_double, C.c_int, _P, _P, C.POINTER(C.c_int), C.POINTER(C.c_double), _P]),
    "ptnet_weight_count": (C.c_size_t, [C.c_int]),
    "ptnet_forward": (C.c_int, [_P, C.c_int, _P, C.c_int, _P, _P, _P]),
    "ptnet_loss_grad": (C.c_int, [_P, C.c_int, _P, C.c_int, _P, _P, _P, C.POINTER(C.c_double), _P]),
    "ptnet_layer16": (C.c_int, [_P, _P, C.c_int, C.c_int, _P, _P, _P]),
    "ptnet_forward_tc": (C.c_int, [_P, C.c_int, _P, C.c_int, _P, _P, _P]),
    "ptnet_adam": (C.c_int, [C.c_size_t, _P, _P, _P, _P, C.c_int, C.c_double, _P]),
    "dfl_inverse_iteration": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.c_int, _P, _P]),
}

_lib = None


def lib():
    """Load libdwsolve.so (built in-tree by build.py); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built: run `python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(LIB_PATH)
        missing = [n for n in _SIGNATURES if not hasattr(L, n)]
        if missing:
            raise RuntimeError(f"{LIB_PATH} lacks exported symbols {missing}")
        for name, (res, args) in _SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def dw_launch_count() -> int:
    return int(lib().dw_launch_count())


def exported_symbols():
    return list(_SIGNATURES)


def _check(rc, ok=(DW_OK,)):
    if rc not in ok:
        raise DwError(rc, lib().dw_last_error().decode())
    return rc


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        return C.c_void_p(t.data_ptr())
    return C.c_void_p(t)


def _stream(stream):
    if stream is None:
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(stream)


def _as_f64(t: torch.Tensor) -> torch.Tensor:
    """complex128 tensors are passed as interleaved doubles."""
    if t.dtype == torch.complex128:
        t = torch.view_as_real(t)
    assert t.dtype == torch.float64 and t.is_contiguous()
    return t


# --------------------------------------------------------------------------- handles
class Ctx:
    def __init__(self, handle, L, params):
        self.handle = handle
        self.L = tuple(L)
        self.V = int(lib().dw_volume(handle))
        self.params = params

    def field_bytes(self, prec):
        return int(lib().dw_field_bytes(self.handle, prec))

    def empty_field(self, prec, nrhs=1, device="cuda"):
        dt = torch.float64 if prec == DW_F64 else torch.float32
        return torch.empty(nrhs * self.V * 24, dtype=dt, device=device)

    def __del__(self):
        try:
            if self.handle:
                lib().dw_destroy(self.handle)
                self.handle = None
        except Exception:
            pass


class Dfl:
    def __init__(self, handle, info):
        self.handle = handle
        self.info = info
        nb, ns = C.c_int(), C.c_int()
        lib().dfl_dims(handle, C.byref(nb), C.byref(ns))
        self.Nb, self.Ns = nb.value, ns.value

    def __del__(self):
        try:
            if self.handle:
                lib().dfl_destroy(self.handle)
                self.handle = None
        except Exception:
            pass


def dw_create(L, m0, csw, links_host: torch.Tensor, sap_bs=(4, 4, 4, 4), antiperiodic=True) -> Ctx:
    p = DwParams()
    p.L = (C.c_int * 4)(*L)
    p.m0, p.csw, p.antiperiodic = float(m0), float(csw), int(bool(antiperiodic))
    p.sap_bs = (C.c_int * 4)(*sap_bs)
    links = _as_f64(links_host.detach().to("cpu").contiguous())
    h = C.c_void_p()
    _check(lib().dw_create(C.byref(p), _ptr(links), C.byref(h)))
    return Ctx(h, L, p)


def dw_release_workspace(ctx: Ctx):
    _check(lib().dw_release_workspace(ctx.handle))


def dw_pack(ctx: Ctx, prec, nrhs, canon_dev, packed_dev, stream=None):
    _check(lib().dw_pack(ctx.handle, prec, nrhs, _ptr(_as_f64(canon_dev)), _ptr(packed_dev), _stream(stream)))


def dw_unpack(ctx: Ctx, prec, nrhs, packed_dev, canon_dev, stream=None):
    _check(lib().dw_unpack(ctx.handle, prec, nrhs, _ptr(packed_dev), _ptr(_as_f64(canon_dev)), _stream(stream)))


def dw_apply(ctx: Ctx, prec, op, nrhs, in_dev, out_dev, stream=None):
    _check(lib().dw_apply(ctx.handle, prec, op, nrhs, _ptr(in_dev), _ptr(out_dev), _stream(stream)))


def dw_apply_schur_static(ctx: Ctx, prec, in_dev, out_dev, stream=None):
    """Schur complement of one packed field without any allocation (fixed 16 MiB device array)."""
    _check(lib().dw_apply_schur_static(ctx.handle, prec, _ptr(in_dev), _ptr(out_dev), _stream(stream)))


def sap_precondition(ctx: Ctx, prec, ncy, nmr, nrhs, rho_dev, xi_dev, stream=None):
    _check(lib().sap_precondition(ctx.handle, prec, ncy, nmr, nrhs, _ptr(rho_dev), _ptr(xi_dev), _stream(stream)))


def deflation_build(ctx: Ctx, bs, Ns, n_inv, ncy, nmr, start_canon_dev, basis_prec=DW_BF16, iter_prec=DW_F32,
                    cond_max=1e8, net_weights=None, net_k0=2, net_judge=0.95, net_channels=16, boot_steps=0,
                    boot_tol=1e-2, boot_nmx=16):
    p = DflParams()
    p.boot_steps, p.boot_tol, p.boot_nmx = int(boot_steps), float(boot_tol), int(boot_nmx)
    p.bs = (C.c_int * 4)(*bs)
    p.Ns, p.n_inv, p.ncy, p.nmr = Ns, n_inv, ncy, nmr
    p.basis_prec, p.iter_prec, p.cond_max = basis_prec, iter_prec, float(cond_max)
    p.net_weights = _ptr(net_weights).value if net_weights is not None else None
    p.net_channels, p.net_k0, p.net_judge = int(net_channels), int(net_k0), float(net_judge)
    info = DflInfo()
    h = C.c_void_p()
    rc = _check(lib().deflation_build(ctx.handle, C.byref(p), _ptr(_as_f64(start_canon_dev)), C.byref(h),
                                      C.byref(info)), ok=(DW_OK, DW_ILLCOND))
    d = Dfl(h, info)
    d.status = rc
    return d


def dfl_retarget(src: Dfl, ctx: Ctx) -> Dfl:
    info = DflInfo()
    h = C.c_void_p()
    rc = _check(lib().dfl_retarget(src.handle, ctx.handle, C.byref(h), C.byref(info)), ok=(DW_OK, DW_ILLCOND))
    d = Dfl(h, info)
    d.status = rc
    return d


def dfl_save(d: Dfl, path):
    _check(lib().dfl_save(d.handle, str(path).encode()))


def dfl_load(ctx: Ctx, path) -> Dfl:
    info = DflInfo()
    h = C.c_void_p()
    rc = _check(lib().dfl_load(ctx.handle, str(path).encode(), C.byref(h), C.byref(info)), ok=(DW_OK, DW_ILLCOND))
    d = Dfl(h, info)
    d.status = rc
    return d


def dfl_restrict(d: Dfl, prec, psi_packed, c_dev, stream=None):
    _check(lib().dfl_restrict(d.handle, prec, _ptr(psi_packed), _ptr(c_dev), _stream(stream)))


def dfl_prolong(d: Dfl, prec, c_dev, psi_packed, stream=None):
    _check(lib().dfl_prolong(d.handle, prec, _ptr(c_dev), _ptr(psi_packed), _stream(stream)))


def dfl_basis_export(d: Dfl, canon_dev, stream=None):
    _check(lib().dfl_basis_export(d.handle, _ptr(_as_f64(canon_dev)), _stream(stream)))


def little_apply(d: Dfl, v_dev, w_dev, stream=None):
    _check(lib().little_apply(d.handle, _ptr(_as_f64(v_dev)), _ptr(_as_f64(w_dev)), _stream(stream)))


def little_dirac_solve(d: Dfl, prec, w_dev, v_dev, tol, maxit, stream=None):
    it, rr = C.c_int(), C.c_double()
    rc = _check(lib().little_dirac_solve(d.handle, prec, _ptr(w_dev), _ptr(v_dev), float(tol), int(maxit),
                                         C.byref(it), C.byref(rr), _stream(stream)), ok=(DW_OK, DW_ENOTCONV))
    return rc, it.value, rr.value


def little_dirac_solve_batch(d: Dfl, prec, nrhs, w_dev, v_dev, tol, maxit, stream=None):
    it, rr = (C.c_int * nrhs)(), (C.c_double * nrhs)()
    rc = _check(lib().little_dirac_solve_batch(d.handle, prec, int(nrhs), _ptr(w_dev), _ptr(v_dev), float(tol),
                                               int(maxit), it, rr, _stream(stream)), ok=(DW_OK, DW_ENOTCONV))
    return rc, list(it), list(rr)


def sol_params(tol=1e-10, nkv=16, nmx=2000, ncy=4, nmr=4, mixed=1, inner_rtol=1e-5, little_tol_out=1e-12,
               little_tol_in=1e-6, little_tol_cap=1e-1, little_nkv=24, little_maxit=2000) -> SolParams:
    p = SolParams()
    p.tol, p.nkv, p.nmx, p.ncy, p.nmr, p.mixed = tol, nkv, nmx, ncy, nmr, mixed
    p.inner_rtol, p.little_tol_out, p.little_tol_in, p.little_tol_cap = inner_rtol, little_tol_out, little_tol_in, \
        little_tol_cap
    p.little_nkv, p.little_maxit = little_nkv, little_maxit
    return p


def gcr_solve(ctx: Ctx, d, params: SolParams, nrhs, eta_dev, psi_dev, stream=None):
    infos = (SolInfo * nrhs)()
    rc = _check(lib().gcr_solve(ctx.handle, d.handle if d is not None else None, C.byref(params), nrhs,
                                _ptr(_as_f64(eta_dev)), _ptr(_as_f64(psi_dev)), infos, _stream(stream)),
                ok=(DW_OK, DW_ENOTCONV))
    return rc, [infos[i] for i in range(nrhs)]


def cgnr_solve(ctx: Ctx, tol, maxit, eta_dev, psi_dev, stream=None):
    it, rr = C.c_int(), C.c_double()
    rc = _check(lib().cgnr_solve(ctx.handle, float(tol), int(maxit), _ptr(_as_f64(eta_dev)), _ptr(_as_f64(psi_dev)),
                                 C.byref(it), C.byref(rr), _stream(stream)), ok=(DW_OK, DW_ENOTCONV))
    return rc, it.value, rr.value


def bicgstab_solve(ctx: Ctx, tol, maxit, eta_dev, psi_dev, stream=None):
    it, rr = C.c_int(), C.c_double()
    rc = _check(lib().bicgstab_solve(ctx.handle, float(tol), int(maxit), _ptr(_as_f64(eta_dev)), _ptr(_as_f64(psi_dev)),
                                     C.byref(it), C.byref(rr), _stream(stream)), ok=(DW_OK, DW_ENOTCONV))
    return rc, it.value, rr.value


def lowmodes_solve(ctx: Ctx, nev, nbuf, start_dev, modes_dev, degree=24, tol=1e-8, maxit=100, prec=DW_F64,
                   stream=None):
    ev, rs, it = (C.c_double * nev)(), (C.c_double * nev)(), C.c_int()
    rc = _check(lib().lowmodes_solve(ctx.handle, int(nev), int(nbuf), int(degree), float(tol), int(maxit), int(prec),
                                     _ptr(_as_f64(start_dev)), _ptr(_as_f64(modes_dev)), ev, rs, C.byref(it),
                                     _stream(stream)), ok=(DW_OK, DW_ENOTCONV))
    return rc, list(ev), list(rs), it.value


def dfl_deficits(d: Dfl, fields_dev, stream=None):
    nf = fields_dev.shape[0]
    eps = (C.c_double * nf)()
    _check(lib().dfl_deficits(d.handle, int(nf), _ptr(_as_f64(fields_dev)), eps, _stream(stream)))
    return list(eps)


def dw_autotune(ctx: Ctx, nrhs=1) -> dict:
    import json
    buf = C.create_string_buffer(1024)
    _check(lib().dw_autotune(ctx.handle, int(nrhs), buf, 1024))
    return json.loads(buf.value.decode())


def dfl_autotune(d: Dfl) -> dict:
    import json
    buf = C.create_string_buffer(1024)
    _check(lib().dfl_autotune(d.handle, buf, 1024))
    return json.loads(buf.value.decode())


def ptnet_weight_count(channels=16) -> int:
    return int(lib().ptnet_weight_count(int(channels)))


def ptnet_forward(ctx: Ctx, weights, nf, x, y, channels=16, stream=None):
    _check(lib().ptnet_forward(ctx.handle, int(channels), _ptr(weights), int(nf), _ptr(x), _ptr(y),
                               _stream(stream)))


def ptnet_layer16(ctx: Ctx, W, adjoint, tensor_cores, x, y, stream=None):
    _check(lib().ptnet_layer16(ctx.handle, _ptr(W), int(adjoint), int(tensor_cores), _ptr(x), _ptr(y), _stream(stream)))


def ptnet_forward_tc(ctx: Ctx, weights, nf, x, y, channels=16, stream=None):
    _check(lib().ptnet_forward_tc(ctx.handle, int(channels), _ptr(weights), int(nf), _ptr(x), _ptr(y),
                                  _stream(stream)))


def ptnet_loss_grad(ctx: Ctx, weights, nf, x, y, grad, channels=16, stream=None) -> float:
    loss = C.c_double()
    _check(lib().ptnet_loss_grad(ctx.handle, int(channels), _ptr(weights), int(nf), _ptr(x), _ptr(y), _ptr(grad),
                                 C.byref(loss), _stream(stream)))
    return loss.value


def ptnet_adam(weights, grad, m, v, step, lr, stream=None):
    n = weights.numel() // 2 if weights.dtype == torch.float32 else weights.numel()
    _check(lib().ptnet_adam(n, _ptr(weights), _ptr(grad), _ptr(m), _ptr(v), int(step), float(lr), _stream(stream)))


def dfl_inverse_iteration(ctx: Ctx, ncy, nmr, nsteps, nf, fields, stream=None):
    _check(lib().dfl_inverse_iteration(ctx.handle, int(ncy), int(nmr), int(nsteps), int(nf), _ptr(fields),
                                       _stream(stream)))
