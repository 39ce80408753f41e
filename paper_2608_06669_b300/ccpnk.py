"""Python binding of libccpnk (include/ccpnk.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts numpy arrays or torch
tensors to pointers, allocates outputs of the matching kind and turns status codes into
exceptions. There is no CPU fallback: if libccpnk.so is missing the first call raises.

Arrays: fock (n, n), B (naux, n, n), t1 (o, v), t2 (o, o, v, v), all float64, C-contiguous.
Inputs may be numpy arrays (host) or torch tensors on the CPU or on the context's GPU;
outputs follow the kind of the first amplitude input (torch CUDA in, torch CUDA out).
"""
from __future__ import annotations

import ctypes
import os
import weakref

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libccpnk.so")

CC_OK, CC_PENDING = 0, 1
STATUS = {-1: "CC_ERR_INVALID", -2: "CC_ERR_OOM", -3: "CC_ERR_NOT_CONVERGED", -4: "CC_ERR_DIVERGED",
          -5: "CC_ERR_CUDA", -6: "CC_ERR_TIMEOUT", -7: "CC_ERR_CANCELLED"}
OPTION = {"stage_cache_bytes": 1, "wait_limit_ns": 2, "graphs": 3, "emu_chunk": 4, "ladder_pack": 5, "emu_onchip": 6}
PREC = {"fp64": 0, "tf32": 1, "bf16x3": 2, "tf32x3": 3, "df64": 4, "fp64emu": 5}
METHOD = {"fp_diis": 0, "nk": 1, "pnk": 2, "ink": 3}


class CCError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class SolveOpts(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int), ("prec", ctypes.c_int), ("tol", ctypes.c_double),
                ("max_outer", ctypes.c_int), ("m_max", ctypes.c_int), ("gamma", ctypes.c_double),
                ("alpha", ctypes.c_double), ("eta_max", ctypes.c_double), ("level_shift", ctypes.c_double),
                ("diis_size", ctypes.c_int), ("jvp_fd", ctypes.c_int), ("inner_rtol", ctypes.c_double),
                ("inner_max", ctypes.c_int), ("af_direct", ctypes.c_int), ("verbose", ctypes.c_int),
                ("ccd", ctypes.c_int), ("max_seconds", ctypes.c_double), ("outer_prec", ctypes.c_int)]


class Report(ctypes.Structure):
    _fields_ = [("energy", ctypes.c_double), ("res_norm", ctypes.c_double), ("newton_iters", ctypes.c_int),
                ("residual_evals", ctypes.c_int), ("jvps", ctypes.c_int), ("af_applies", ctypes.c_int),
                ("krylov_iters", ctypes.c_int), ("status", ctypes.c_int), ("seconds", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib() -> ctypes.CDLL:
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2608_06669_b300.build`")
        L = ctypes.CDLL(LIB_PATH)
        vp, i, d, sz, u64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t, ctypes.c_uint64
        pp = ctypes.POINTER(ctypes.c_void_p)
        sig = {
            "cc_solve_opts_default": (None, [ctypes.POINTER(SolveOpts), i, i]),
            "cc_ctx_create": (i, [pp, i, sz, vp]),
            "cc_ctx_destroy": (None, [vp]),
            "cc_last_error": (ctypes.c_char_p, [vp]),
            "cc_ctx_device_bytes": (sz, [vp]),
            "cc_ctx_launches": (u64, [vp]),
            "cc_ctx_launch_calls": (u64, [vp]),
            "cc_ctx_set_option": (i, [vp, i, ctypes.c_longlong]),
            "cc_ctx_selftest_wait": (i, [vp]),
            "cc_probe_fma_rate": (i, [i, i, ctypes.POINTER(d)]),
            "cc_ctx_profile": (i, [vp, i]),
            "cc_ctx_profile_get": (i, [vp, ctypes.c_char_p, ctypes.POINTER(u64), ctypes.POINTER(d), ctypes.POINTER(d)]),
            "cc_ctx_profile_list": (i, [vp, ctypes.c_char_p, sz, ctypes.POINTER(sz)]),
            "cc_sys_create": (i, [vp, i, i, i, vp, vp, pp]),
            "cc_sys_destroy": (None, [vp]),
            "cc_residual": (i, [vp, vp, vp, vp, vp, vp, ctypes.POINTER(d), i]),
            "cc_jvp": (i, [vp, vp, vp, vp, vp, vp, vp, vp, i]),
            "cc_jvp_multi": (i, [vp, vp, vp, vp, i, vp, vp, vp, vp, i]),
            "cc_apply_AF": (i, [vp, vp, vp, vp, vp, vp, i, i]),
            "cc_solve": (i, [vp, vp, ctypes.POINTER(SolveOpts), vp, vp, i, ctypes.POINTER(Report)]),
            "cc_solve_batch": (i, [vp, i, ctypes.POINTER(vp), ctypes.POINTER(SolveOpts), ctypes.POINTER(vp),
                                   ctypes.POINTER(vp), ctypes.POINTER(Report)]),
            "cc_energy_noalloc": (i, [vp, vp, vp, vp, vp]),
            "cc_server_create": (i, [pp, i, sz, i]),
            "cc_server_destroy": (None, [vp]),
            "cc_serve_submit": (i, [vp, i, i, i, vp, vp, ctypes.POINTER(SolveOpts), ctypes.POINTER(u64)]),
            "cc_serve_poll": (i, [vp, u64, ctypes.POINTER(Report), vp, vp]),
            "cc_serve_cancel": (i, [vp, u64]),
            "cc_server_set_grouping": (i, [vp, i]),
            "cc_server_set_policy": (i, [vp, i]),
            "cc_serve_times": (i, [vp, u64, ctypes.POINTER(d), ctypes.POINTER(d), ctypes.POINTER(d)]),
            "cc_server_stats": (i, [vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(sz)]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


# ---------------------------------------------------------------------------
# array marshalling
# ---------------------------------------------------------------------------
def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x, keep: list):
    """Pointer to a float64 C-contiguous buffer (numpy or torch); copies are kept alive in keep."""
    if x is None:
        return None
    if _is_torch(x):
        import torch

        if x.dtype != torch.float64 or not x.is_contiguous():
            x = x.to(torch.float64).contiguous()
        keep.append(x)
        return ctypes.c_void_p(x.data_ptr())
    a = np.ascontiguousarray(x, dtype=np.float64)
    keep.append(a)
    return ctypes.c_void_p(a.ctypes.data)


def _empty_like_kind(ref, shape):
    if _is_torch(ref):
        import torch

        return torch.empty(shape, dtype=torch.float64, device=ref.device)
    return np.empty(shape, dtype=np.float64)


def _check(ctx, status):
    if status < 0:
        raise CCError(status, lib().cc_last_error(ctx).decode())
    return status


def _prec(p) -> int:
    return PREC[p] if isinstance(p, str) else int(p)


# ---------------------------------------------------------------------------
# objects
# ---------------------------------------------------------------------------
class Context:
    """A device context (cc_ctx). stream: 'torch' to run on torch's current stream, None for
    a private stream, or a raw cudaStream_t integer."""

    def __init__(self, device: int = 0, mem_budget: int = 0, stream="torch"):
        L = lib()
        s = None
        if stream == "torch":
            import torch

            s = ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)
        elif stream is not None:
            s = ctypes.c_void_p(int(stream))
        h = ctypes.c_void_p()
        st = L.cc_ctx_create(ctypes.byref(h), device, mem_budget, s)
        if st < 0:
            raise CCError(st, "cc_ctx_create failed")
        self.h = h
        self.device = device
        self.systems = weakref.WeakSet()  # closed before the context is

    @property
    def device_bytes(self) -> int:
        return int(lib().cc_ctx_device_bytes(self.h))

    @property
    def launches(self) -> int:
        return int(lib().cc_ctx_launches(self.h))

    @property
    def launch_calls(self) -> int:
        return int(lib().cc_ctx_launch_calls(self.h))

    def set_option(self, name: str, value: int):
        """cc_ctx_set_option: 'stage_cache_bytes' (-1 default, 0 off), 'wait_limit_ns' or 'graphs' (0/1)."""
        _check(self.h, lib().cc_ctx_set_option(self.h, OPTION[name], int(value)))

    def selftest_wait(self) -> int:
        """cc_ctx_selftest_wait: the status of one bounded wait that is made to give up
        (CC_ERR_TIMEOUT, -6, when the bound works)."""
        return int(lib().cc_ctx_selftest_wait(self.h))

    def profile(self, enable: bool = True, all_contractions: bool = False):
        """Turns the kernel timer on (clearing its records) or off. On, it times the ladder
        GEMMs; with all_contractions also every other contraction, under its index labels."""
        _check(self.h, lib().cc_ctx_profile(self.h, (2 if all_contractions else 1) if enable else 0))

    def profile_get(self, tag: str):
        """(launches, total_ms, flops) recorded for a tag since profile(True)."""
        n, ms, fl = ctypes.c_uint64(), ctypes.c_double(), ctypes.c_double()
        _check(self.h, lib().cc_ctx_profile_get(self.h, tag.encode(), ctypes.byref(n), ctypes.byref(ms),
                                                ctypes.byref(fl)))
        return int(n.value), float(ms.value), float(fl.value)

    def profile_list(self):
        """{tag: (launches, total_ms, flops)} for every tag recorded since profile(True)."""
        need = ctypes.c_size_t()
        _check(self.h, lib().cc_ctx_profile_list(self.h, None, 0, ctypes.byref(need)))
        buf = ctypes.create_string_buffer(need.value)
        _check(self.h, lib().cc_ctx_profile_list(self.h, buf, need.value, None))
        out = {}
        for line in buf.value.decode().splitlines():
            tag, n, ms, fl = line.split("\t")
            out[tag] = (int(n), float(ms), float(fl))
        return out

    def close(self):
        if getattr(self, "h", None):
            for s in list(getattr(self, "systems", ())):
                s.close()
            lib().cc_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class System:
    """A problem resident on the device (cc_sys): copies fock (n, n) and B (naux, n, n)."""

    def __init__(self, ctx: Context, o: int, v: int, naux: int, fock, B):
        keep = []
        h = ctypes.c_void_p()
        if not getattr(ctx, "h", None):
            raise CCError(-1, "the context is closed")
        _check(ctx.h, lib().cc_sys_create(ctx.h, o, v, naux, _ptr(fock, keep), _ptr(B, keep), ctypes.byref(h)))
        self.ctx, self.h, self.o, self.v, self.naux = ctx, h, o, v, naux
        ctx.systems.add(self)

    @classmethod
    def from_synth(cls, ctx: Context, s):
        return cls(ctx, s.o, s.v, s.naux, s.fock, s.B)

    def close(self):
        if getattr(self, "h", None):
            lib().cc_sys_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- the hot path -------------------------------------------------------
    def residual(self, t1, t2, prec="fp64"):
        """(r1, r2, E): R(t) and the correlation energy."""
        keep = []
        r1 = _empty_like_kind(t1, (self.o, self.v))
        r2 = _empty_like_kind(t1, (self.o, self.o, self.v, self.v))
        e = ctypes.c_double()
        _check(self.ctx.h, lib().cc_residual(self.ctx.h, self.h, _ptr(t1, keep), _ptr(t2, keep), _ptr(r1, keep),
                                             _ptr(r2, keep), ctypes.byref(e), _prec(prec)))
        return r1, r2, e.value

    def jvp(self, t1, t2, d1, d2, prec="fp64"):
        """(j1, j2) = J(t) d."""
        keep = []
        j1 = _empty_like_kind(t1, (self.o, self.v))
        j2 = _empty_like_kind(t1, (self.o, self.o, self.v, self.v))
        _check(self.ctx.h, lib().cc_jvp(self.ctx.h, self.h, _ptr(t1, keep), _ptr(t2, keep), _ptr(d1, keep),
                                        _ptr(d2, keep), _ptr(j1, keep), _ptr(j2, keep), _prec(prec)))
        return j1, j2

    def jvp_multi(self, t1, t2, D1, D2, prec="fp64"):
        """(J1, J2) with J[k] = J(t) D[k] for the k = 0..ndir-1 stacked directions."""
        keep = []
        nd = int(D1.shape[0])
        J1 = _empty_like_kind(t1, (nd, self.o, self.v))
        J2 = _empty_like_kind(t1, (nd, self.o, self.o, self.v, self.v))
        _check(self.ctx.h, lib().cc_jvp_multi(self.ctx.h, self.h, _ptr(t1, keep), _ptr(t2, keep), nd, _ptr(D1, keep),
                                              _ptr(D2, keep), _ptr(J1, keep), _ptr(J2, keep), _prec(prec)))
        return J1, J2

    def apply_AF(self, x1, x2, inverse: int = 0, prec="fp64"):
        """A_F x (inverse=0), A_F^{-1} x by inner GMRES (1) or in the Fock eigenbasis (2)."""
        keep = []
        y1 = _empty_like_kind(x1, (self.o, self.v))
        y2 = _empty_like_kind(x1, (self.o, self.o, self.v, self.v))
        _check(self.ctx.h, lib().cc_apply_AF(self.ctx.h, self.h, _ptr(x1, keep), _ptr(x2, keep), _ptr(y1, keep),
                                             _ptr(y2, keep), int(inverse), _prec(prec)))
        return y1, y2

    def solve(self, method="pnk", prec="fp64", t1=None, t2=None, **kw):
        """Solves R(t) = 0; returns (t1, t2, report dict). Keywords override cc_solve_opts fields."""
        opts = default_opts(method, prec, **kw)
        keep = []
        ref = t1 if t1 is not None else np.empty(0)
        o1 = _empty_like_kind(ref, (self.o, self.v))
        o2 = _empty_like_kind(ref, (self.o, self.o, self.v, self.v))
        use_guess = t1 is not None
        if use_guess:
            o1[...] = t1
            o2[...] = t2
        rep = Report()
        st = lib().cc_solve(self.ctx.h, self.h, ctypes.byref(opts), _ptr(o1, keep), _ptr(o2, keep),
                            int(use_guess), ctypes.byref(rep))
        if st not in (0, -3, -4):
            _check(self.ctx.h, st)
        d = rep.as_dict()
        d["status_code"] = st
        return o1, o2, d


def solve_batch(ctx: Context, systems, method="pnk", prec="fp64", **kw):
    """cc_solve_batch: solves the systems (of one context) together in lockstep; returns a list
    of (t1, t2, report dict) in the systems' order, amplitudes as numpy arrays."""
    n = len(systems)
    opts = default_opts(method, prec, **kw)
    outs = [(np.empty((s.o, s.v)), np.empty((s.o, s.o, s.v, s.v))) for s in systems]
    hs = (ctypes.c_void_p * n)(*[s.h for s in systems])
    p1 = (ctypes.c_void_p * n)(*[o[0].ctypes.data for o in outs])
    p2 = (ctypes.c_void_p * n)(*[o[1].ctypes.data for o in outs])
    reps = (Report * n)()
    _check(ctx.h, lib().cc_solve_batch(ctx.h, n, hs, ctypes.byref(opts), p1, p2, reps))
    res = []
    for k in range(n):
        d = reps[k].as_dict()
        d["status_code"] = d["status"]
        res.append((outs[k][0], outs[k][1], d))
    return res


class Server:
    """The continuous-batching server (cc_server): submit() returns a ticket at once; poll()
    returns None while the request waits or runs, then (t1, t2, report dict)."""

    def __init__(self, device: int = 0, mem_budget: int = 0, max_slots: int = 4):
        h = ctypes.c_void_p()
        st = lib().cc_server_create(ctypes.byref(h), device, mem_budget, max_slots)
        if st < 0:
            raise CCError(st, "cc_server_create failed")
        self.h = h
        self.shapes = {}

    def submit(self, o, v, naux, fock, B, method="pnk", prec="fp64", **kw) -> int:
        keep = []
        opts = default_opts(method, prec, **kw)
        t = ctypes.c_uint64()
        st = lib().cc_serve_submit(self.h, o, v, naux, _ptr(np.asarray(fock), keep), _ptr(np.asarray(B), keep),
                                   ctypes.byref(opts), ctypes.byref(t))
        if st < 0:
            raise CCError(st, "cc_serve_submit failed")
        self.shapes[t.value] = (o, v)
        return t.value

    def poll(self, ticket: int):
        o, v = self.shapes[ticket]
        t1 = np.empty((o, v))
        t2 = np.empty((o, o, v, v))
        rep = Report()
        st = lib().cc_serve_poll(self.h, ticket, ctypes.byref(rep), ctypes.c_void_p(t1.ctypes.data),
                                 ctypes.c_void_p(t2.ctypes.data))
        if st == CC_PENDING:
            return None
        d = rep.as_dict()
        d["status_code"] = st
        return t1, t2, d

    def set_grouping(self, group_max: int):
        """cc_server_set_grouping: a slot solves up to group_max compatible requests together."""
        st = lib().cc_server_set_grouping(self.h, int(group_max))
        if st < 0:
            raise CCError(st, "cc_server_set_grouping failed")

    def set_policy(self, policy: str):
        """cc_server_set_policy: 'fifo' or 'shortest_first'."""
        st = lib().cc_server_set_policy(self.h, {"fifo": 0, "shortest_first": 1}[policy])
        if st < 0:
            raise CCError(st, "cc_server_set_policy failed")

    def cancel(self, ticket: int) -> int:
        """cc_serve_cancel: drops a waiting request or stops a running one."""
        return int(lib().cc_serve_cancel(self.h, ticket))

    def times(self, ticket: int):
        a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        lib().cc_serve_times(self.h, ticket, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
        return a.value, b.value, c.value

    def stats(self):
        r, q, m = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        b = ctypes.c_size_t()
        lib().cc_server_stats(self.h, ctypes.byref(r), ctypes.byref(q), ctypes.byref(m), ctypes.byref(b))
        return {"running": r.value, "queued": q.value, "max_running": m.value, "bytes_admitted": b.value}

    def close(self):
        if getattr(self, "h", None):
            lib().cc_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def probe_fma_rate(device: int = 0, fp64: bool = True) -> float:
    """cc_probe_fma_rate: measured FMA throughput of the FP64 (or FP32) pipe in TFLOP/s."""
    r = ctypes.c_double()
    st = lib().cc_probe_fma_rate(device, 1 if fp64 else 0, ctypes.byref(r))
    if st < 0:
        raise CCError(st, "cc_probe_fma_rate failed")
    return r.value


def default_opts(method="pnk", prec="fp64", **kw) -> SolveOpts:
    opts = SolveOpts()
    lib().cc_solve_opts_default(ctypes.byref(opts), METHOD[method] if isinstance(method, str) else int(method),
                                _prec(prec))
    for k, v in kw.items():
        if not hasattr(opts, k):
            raise KeyError(k)
        setattr(opts, k, v)
    return opts
