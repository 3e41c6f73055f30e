"""GB300 (sm_103a) inexact GMRES policy iteration for finite discounted-cost MDPs.

Thin Python binding over the C ABI of libmdpgpu (include/mdpgpu.h).  Each function has the
name of the C entry point it calls and only marshals arguments: numpy arrays go to the
host-pointer entry points, CUDA torch tensors to the *_dev ones.  Every arithmetic step runs
in the library's CUDA kernels; when the library is missing, importing a function raises.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib
from ._lib import (MDP_F32, MDP_F64, MDP_FLAG_HOST_LOOP, MDP_FLAG_NO_WINDOW, MDP_PREC_FP64,  # noqa: F401
                   MDP_FLAG_PC_REBUILD,
                   MDP_PREC_MIXED, MDPError, mdp_opts, mdp_server_opts, mdp_stats)

__all__ = [
    "MDPHandle", "mdp_create_dense", "mdp_create_ell", "bellman_apply", "policy_eval_gmres",
    "ipi_solve", "vi_solve", "pi_solve", "opi_solve", "ipi_vi_solve", "opts", "MDP_PREC_FP64",
    "MDPBatch", "ipi_solve_batch", "MDPServer",
    "MDP_PREC_MIXED", "MDPError", "lib",
]


def lib():
    return _lib.load()


def _is_cuda(x) -> bool:
    return getattr(x, "is_cuda", False)


def _ptr(x):
    """Address of a contiguous numpy array or CUDA tensor (None -> NULL)."""
    if x is None:
        return None
    if _is_cuda(x):
        if not x.is_contiguous():
            raise ValueError("device tensors must be contiguous")
        return C.c_void_p(x.data_ptr())
    if not x.flags["C_CONTIGUOUS"]:
        raise ValueError("host arrays must be C-contiguous")
    return C.c_void_p(x.ctypes.data)


def _check(code, where):
    if code < 0 and code != _lib.MDP_ENOCONV:
        raise MDPError(code, where)
    return code


def _dtype_code(arr) -> int:
    name = str(arr.dtype)
    if name.endswith("float32"):
        return MDP_F32
    if name.endswith("float64"):
        return MDP_F64
    raise TypeError(f"transition data must be float32 or float64, not {arr.dtype}")


class MDPHandle:
    """Owns an mdp_t; destroyed with the object (or explicitly with close())."""

    def __init__(self, ptr, S, A, k, kind, dtype):
        self._p = ptr
        self.S, self.A, self.k, self.kind, self.dtype = S, A, k, kind, dtype

    @property
    def ptr(self):
        if self._p is None:
            raise ValueError("handle is closed")
        return self._p

    def close(self):
        if self._p is not None:
            lib().mdp_destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def device_bytes(self) -> int:
        return int(lib().mdp_device_bytes(self.ptr))

    def set_stream(self, stream) -> None:
        """stream: torch.cuda.Stream, an integer cudaStream_t, or None."""
        s = getattr(stream, "cuda_stream", stream)
        _check(lib().mdp_set_stream(self.ptr, C.c_void_p(s) if s else None), "mdp_set_stream")

    def set_timing(self, on: bool) -> None:
        _check(lib().mdp_set_timing(self.ptr, 1 if on else 0), "mdp_set_timing")

    def set_tuning(self, ell_lanes_sweep: int = 0, ell_lanes_matvec: int = 0) -> None:
        _check(lib().mdp_set_tuning(self.ptr, ell_lanes_sweep, ell_lanes_matvec), "mdp_set_tuning")

    def set_geometry(self, sweep_blocks: int = 0, matvec_blocks: int = 0,
                     krylov_blocks: int = 0) -> None:
        _check(lib().mdp_set_geometry(self.ptr, sweep_blocks, matvec_blocks, krylov_blocks),
               "mdp_set_geometry")


def mdp_create_dense(P, g, gamma: float, mask=None) -> MDPHandle:
    """P[a, s, s'] (A, S, S) float32/float64, g[a, s] (A, S) float64, mask[s, a] uint8."""
    A, S, S2 = P.shape
    if S != S2 or tuple(g.shape) != (A, S):
        raise ValueError("P must be (A, S, S) and g (A, S)")
    h = C.c_void_p()
    fn = lib().mdp_create_dense_dev if _is_cuda(P) else lib().mdp_create_dense
    _check(fn(S, A, _ptr(P), _dtype_code(P), _ptr(g), float(gamma), _ptr(mask), C.byref(h)),
           "mdp_create_dense")
    return MDPHandle(h, S, A, 0, "dense", _dtype_code(P))


def mdp_create_ell(col, val, g, gamma: float, mask=None) -> MDPHandle:
    """col/val[a, s, j] (A, S, k) int32 / float32|float64, g[a, s] (A, S) float64."""
    A, S, k = val.shape
    if tuple(col.shape) != (A, S, k) or tuple(g.shape) != (A, S):
        raise ValueError("col/val must be (A, S, k) and g (A, S)")
    h = C.c_void_p()
    fn = lib().mdp_create_ell_dev if _is_cuda(val) else lib().mdp_create_ell
    _check(fn(S, A, k, _ptr(col), _ptr(val), _dtype_code(val), _ptr(g), float(gamma),
              _ptr(mask), C.byref(h)), "mdp_create_ell")
    return MDPHandle(h, S, A, k, "ell", _dtype_code(val))


def mdp_load_dense(h: MDPHandle, P, g) -> None:
    _check(lib().mdp_load_dense(h.ptr, _ptr(P), _ptr(g)), "mdp_load_dense")


def mdp_load_ell(h: MDPHandle, col, val, g) -> None:
    _check(lib().mdp_load_ell(h.ptr, _ptr(col), _ptr(val), _ptr(g)), "mdp_load_ell")


def mdp_load_dense_async(h: MDPHandle, P, g) -> None:
    """Enqueue the load (arrays must stay alive until the next call on h returns)."""
    _check(lib().mdp_load_dense_async(h.ptr, _ptr(P), _ptr(g)), "mdp_load_dense_async")


def mdp_load_ell_async(h: MDPHandle, col, val, g) -> None:
    """Enqueue the load (arrays must stay alive until the next call on h returns)."""
    _check(lib().mdp_load_ell_async(h.ptr, _ptr(col), _ptr(val), _ptr(g)), "mdp_load_ell_async")


def opts(**kw) -> mdp_opts:
    """mdp_opts with the library defaults, overridden by keyword (v0 must stay alive)."""
    o = lib().mdp_opts_default()
    for key, val in kw.items():
        if key == "v0":
            o.v0 = C.cast(_ptr(val), C.POINTER(C.c_double)) if val is not None else None
        elif key == "precision" and isinstance(val, str):
            o.precision = MDP_PREC_MIXED if val == "mixed" else MDP_PREC_FP64
        else:
            setattr(o, key, val)
    return o


def _prec(p) -> int:
    if isinstance(p, str):
        return MDP_PREC_MIXED if p == "mixed" else MDP_PREC_FP64
    return int(p)


def _new_like(h: MDPHandle, device, dtype):
    if device:
        import torch
        tdt = torch.float64 if dtype == "f64" else torch.int32
        return torch.empty(h.S, dtype=tdt, device="cuda")
    return np.empty(h.S, dtype=np.float64 if dtype == "f64" else np.int32)


def bellman_apply(h: MDPHandle, v, precision=MDP_PREC_MIXED, margin: bool = False):
    """One Bellman sweep at v -> (Tv, pi, ||Tv - v||_inf[, margin])."""
    dev = _is_cuda(v)
    Tv, pi = _new_like(h, dev, "f64"), _new_like(h, dev, "i32")
    res = C.c_double(0.0)
    if dev:
        mg = _new_like(h, True, "f64") if margin else None
        _check(lib().bellman_apply_dev(h.ptr, _ptr(v), _ptr(Tv), _ptr(pi), _ptr(mg),
                                       C.cast(C.pointer(res), C.c_void_p), _prec(precision)),
               "bellman_apply_dev")
        return (Tv, pi, res.value, mg) if margin else (Tv, pi, res.value)
    if margin:
        raise ValueError("margin output is available through device tensors only")
    v = np.ascontiguousarray(v, dtype=np.float64)
    _check(lib().bellman_apply(h.ptr, _ptr(v), _ptr(Tv), _ptr(pi),
                               C.cast(C.pointer(res), C.c_void_p), _prec(precision)),
           "bellman_apply")
    return Tv, pi, res.value


def policy_eval_gmres(h: MDPHandle, pi, v0=None, target_inf: float = 1e-10, o=None):
    """GMRES(W) policy evaluation -> (V, stats dict)."""
    dev = _is_cuda(pi)
    o = o or opts()
    out = _new_like(h, dev, "f64")
    st = mdp_stats()
    fn = lib().policy_eval_gmres_dev if dev else lib().policy_eval_gmres
    if not dev:
        pi = np.ascontiguousarray(pi, dtype=np.int32)
        v0 = None if v0 is None else np.ascontiguousarray(v0, dtype=np.float64)
    _check(fn(h.ptr, _ptr(pi), _ptr(v0), float(target_inf), C.byref(o), _ptr(out), C.byref(st)),
           "policy_eval_gmres")
    return out, st.as_dict()


def _solve(name: str, h: MDPHandle, o=None, device: bool = False, v_out=None, pi_out=None):
    o = o or opts()
    v = v_out if v_out is not None else _new_like(h, device, "f64")
    pi = pi_out if pi_out is not None else _new_like(h, device, "i32")
    st = mdp_stats()
    dev = _is_cuda(v)
    fn = getattr(lib(), name + ("_dev" if dev else ""))
    _check(fn(h.ptr, C.byref(o), _ptr(v), _ptr(pi), C.byref(st)), name)
    return v, pi, st.as_dict()


def ipi_solve(h, o=None, device=False, v_out=None, pi_out=None):
    """iGMRES-PI (Alg. 2) -> (v = T(V_K), pi, stats)."""
    return _solve("ipi_solve", h, o, device, v_out, pi_out)


def vi_solve(h, o=None, device=False, v_out=None, pi_out=None):
    return _solve("vi_solve", h, o, device, v_out, pi_out)


def pi_solve(h, o=None, device=False, v_out=None, pi_out=None):
    return _solve("pi_solve", h, o, device, v_out, pi_out)


def opi_solve(h, o=None, device=False, v_out=None, pi_out=None):
    return _solve("opi_solve", h, o, device, v_out, pi_out)


def ipi_vi_solve(h, o=None, device=False, v_out=None, pi_out=None):
    """Inexact PI with VI as the inner solver (Alg. 1) -> (v, pi, stats)."""
    return _solve("ipi_vi_solve", h, o, device, v_out, pi_out)


def from_synth(m, device: bool = False) -> MDPHandle:
    """Create a handle from an object with the fields of mdp_synth.SynthMDP."""
    mask = None if m.mask is None else np.ascontiguousarray(m.mask, dtype=np.uint8)
    g = np.ascontiguousarray(m.g, dtype=np.float64)
    if device:
        import torch
        cv = lambda x: None if x is None else torch.from_numpy(np.ascontiguousarray(x)).cuda()
        if m.kind == "dense":
            return mdp_create_dense(cv(m.P), cv(g), m.gamma, cv(mask))
        return mdp_create_ell(cv(m.col), cv(m.val), cv(g), m.gamma, cv(mask))
    if m.kind == "dense":
        return mdp_create_dense(np.ascontiguousarray(m.P), g, m.gamma, mask)
    return mdp_create_ell(np.ascontiguousarray(m.col, dtype=np.int32),
                          np.ascontiguousarray(m.val), g, m.gamma, mask)


class MDPBatch:
    """mdp_batch_t over ELL handles (mixed precision); keeps the handles alive."""

    def __init__(self, handles, o=None):
        self.handles = list(handles)
        self.n = len(self.handles)
        arr = (C.c_void_p * self.n)(*[h.ptr.value for h in self.handles])
        self._p = C.c_void_p()
        o = o or opts()
        _check(lib().mdp_batch_create(arr, self.n, C.byref(o), C.byref(self._p)),
               "mdp_batch_create")

    @property
    def ptr(self):
        if self._p is None:
            raise ValueError("batch is closed")
        return self._p

    def close(self):
        if self._p is not None:
            lib().mdp_batch_destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream) -> None:
        s = getattr(stream, "cuda_stream", stream)
        _check(lib().mdp_batch_set_stream(self.ptr, C.c_void_p(s) if s else None),
               "mdp_batch_set_stream")

    def tune(self) -> None:
        _check(lib().mdp_batch_tune(self.ptr), "mdp_batch_tune")

    def geometry(self, i: int) -> dict:
        v = [C.c_int32() for _ in range(5)]
        _check(lib().mdp_batch_geometry(self.ptr, i, *[C.byref(x) for x in v]),
               "mdp_batch_geometry")
        keys = ("lanes_sweep", "lanes_matvec", "sweep_blocks", "matvec_blocks", "krylov_blocks")
        return dict(zip(keys, (x.value for x in v)))

    def device_bytes(self) -> int:
        return int(lib().mdp_batch_device_bytes(self.ptr))

    def bellman(self, wait: bool = True):
        """One Bellman sweep of every instance at its current V -> ||T V - V||_inf per
        instance (wait=False only enqueues the launches and returns None)."""
        if not wait:
            _check(lib().mdp_batch_bellman(self.ptr, None), "mdp_batch_bellman")
            return None
        res = np.empty(self.n, dtype=np.float64)
        _check(lib().mdp_batch_bellman(self.ptr, _ptr(res)), "mdp_batch_bellman")
        return res

    def solve(self, v_out=None, pi_out=None, device: bool = False):
        """Solve every instance -> (list of v, list of pi, list of stats dicts, status)."""
        if v_out is None:
            v_out = [_new_like(h, device, "f64") for h in self.handles]
        if pi_out is None:
            pi_out = [_new_like(h, device, "i32") for h in self.handles]
        dev = _is_cuda(v_out[0])
        vp = (C.c_void_p * self.n)(*[_ptr(x).value for x in v_out])
        pp = (C.c_void_p * self.n)(*[_ptr(x).value for x in pi_out])
        st = (mdp_stats * self.n)()
        fn = lib().mdp_batch_solve_dev if dev else lib().mdp_batch_solve
        code = _check(fn(self.ptr, vp, pp, st), "mdp_batch_solve")
        return v_out, pi_out, [s.as_dict() for s in st], code


def ipi_solve_batch(handles, o=None):
    """One-shot batched iGMRES-PI into host arrays -> (vs, pis, stats, status)."""
    n = len(handles)
    arr = (C.c_void_p * n)(*[h.ptr.value for h in handles])
    vs = [np.empty(h.S, dtype=np.float64) for h in handles]
    ps = [np.empty(h.S, dtype=np.int32) for h in handles]
    vp = (C.c_void_p * n)(*[x.ctypes.data for x in vs])
    pp = (C.c_void_p * n)(*[x.ctypes.data for x in ps])
    st = (mdp_stats * n)()
    o = o or opts()
    code = _check(lib().ipi_solve_batch(arr, n, C.byref(o), vp, pp, st), "ipi_solve_batch")
    return vs, ps, [s.as_dict() for s in st], code


class MDPServer:
    """mdp_server_t: continuous batching of iGMRES-PI requests (mixed precision).

    submit() takes ELL data as arrays col/val [A, S, k] (int32 / float32), g [A, S]
    (float64) and output buffers; every array must stay alive (the object keeps references)
    until the request is reported by poll()/drain()."""

    def __init__(self, hbm_budget_bytes=None, max_slots=None, iters_per_launch=None, o=None):
        so = lib().mdp_server_opts_default()
        if hbm_budget_bytes is not None:
            so.hbm_budget_bytes = int(hbm_budget_bytes)
        if max_slots is not None:
            so.max_slots = int(max_slots)
        if iters_per_launch is not None:
            so.iters_per_launch = int(iters_per_launch)
        if o is not None:
            so.solver = o
        self._p = C.c_void_p()
        _check(lib().mdp_server_create(C.byref(so), C.byref(self._p)), "mdp_server_create")
        self._keep = {}
        self.results = {}

    @property
    def ptr(self):
        if self._p is None:
            raise ValueError("server is closed")
        return self._p

    def close(self):
        if self._p is not None:
            lib().mdp_server_destroy(self._p)
            self._p = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, col, val, g, gamma, v_out=None, pi_out=None) -> int:
        A, S, k = val.shape
        if v_out is None:
            v_out = np.empty(S, dtype=np.float64)
        if pi_out is None:
            pi_out = np.empty(S, dtype=np.int32)
        rid = C.c_int64()
        _check(lib().mdp_server_submit(self.ptr, S, A, k, _ptr(col), _ptr(val), _ptr(g),
                                       float(gamma), _ptr(v_out), _ptr(pi_out), C.byref(rid)),
               "mdp_server_submit")
        self._keep[rid.value] = (col, val, g, v_out, pi_out)
        return rid.value

    def poll(self, max_done: int = 1024):
        """Advance; returns [(id, v, pi, stats dict)] of the requests completed since."""
        ids = (C.c_int64 * max_done)()
        st = (mdp_stats * max_done)()
        n = C.c_int32()
        _check(lib().mdp_server_poll(self.ptr, ids, st, max_done, C.byref(n)), "mdp_server_poll")
        out = []
        for i in range(n.value):
            _, _, _, v, pi = self._keep.pop(ids[i])
            out.append((ids[i], v, pi, st[i].as_dict()))
        return out

    def drain(self):
        """Run until every submitted request completed -> the poll() list of all of them."""
        _check(lib().mdp_server_drain(self.ptr), "mdp_server_drain")
        out = []
        while True:
            part = self.poll()
            out.extend(part)
            if not part:
                break
        return out

    def info(self) -> dict:
        a, p, b, l = C.c_int32(), C.c_int32(), C.c_int64(), C.c_int64()
        _check(lib().mdp_server_info(self.ptr, C.byref(a), C.byref(p), C.byref(b), C.byref(l)),
               "mdp_server_info")
        return {"active": a.value, "pending": p.value, "bytes_in_use": b.value, "launches": l.value}


def probe_alu(dtype: str = "f64") -> float:
    """Measured FMA rate of the current GPU in TFLOP/s (mdp_probe_alu), "f64" or "f32"."""
    out = C.c_double(0.0)
    _check(lib().mdp_probe_alu(MDP_F64 if dtype == "f64" else MDP_F32, C.byref(out)),
           "mdp_probe_alu")
    return out.value


def precond_coarse_inverse(h: MDPHandle, pi, block: int):
    """J_c^{-1} of the two-level preconditioner for policy pi (mdp_precond_coarse_inverse)
    -> (inverse as an (nc, nc) float32 array, band half-width in blocks)."""
    pi = np.ascontiguousarray(pi, dtype=np.int32)
    nc, bw = C.c_int64(), C.c_int32()
    _check(lib().mdp_precond_coarse_inverse(h.ptr, _ptr(pi), int(block), None, C.byref(nc),
                                            C.byref(bw)), "mdp_precond_coarse_inverse")
    inv = np.empty((nc.value, nc.value), dtype=np.float32)
    _check(lib().mdp_precond_coarse_inverse(h.ptr, _ptr(pi), int(block), _ptr(inv), C.byref(nc),
                                            C.byref(bw)), "mdp_precond_coarse_inverse")
    return inv, bw.value


# ---------------------------------------------------------------- row-sharded solve
def row_partition(S: int, world: int) -> np.ndarray:
    """Contiguous, balanced row blocks: row_begin[r] = floor(r * S / world), [world + 1]."""
    return np.array([(r * S) // world for r in range(world + 1)], dtype=np.int64)


class ShardComm:
    """Host collectives of ipi_solve_sharded over a torch.distributed process group (CPU
    tensors: gloo; for an NCCL job pass a gloo group made with torch.distributed.new_group).
    Every rank of the group builds one with the same row partition."""

    def __init__(self, row_begin, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.row_begin = np.ascontiguousarray(row_begin, dtype=np.int64)
        if self.row_begin.shape != (self.world + 1,):
            raise ValueError("row_begin must have world + 1 entries")
        self._ag = _lib.ALLGATHER_FN(self._allgather)
        self._ar = _lib.ALLREDUCE_FN(self._allreduce)
        self.c = _lib.mdp_comm(None, self.rank, self.world,
                               self.row_begin.ctypes.data_as(C.POINTER(C.c_int64)),
                               self._ag, self._ar)

    def allgather(self, local: np.ndarray, bytes_per_row: int) -> np.ndarray:
        """Every rank's rows (raw bytes, this rank's in `local`) in row order."""
        import torch
        rb = self.row_begin
        counts = np.diff(rb) * bytes_per_row
        buf = np.zeros(int(counts.max()), dtype=np.uint8)
        buf[:counts[self.rank]] = np.frombuffer(local, dtype=np.uint8, count=int(counts[self.rank]))
        t = torch.from_numpy(buf)
        outs = [torch.empty_like(t) for _ in range(self.world)]
        self.dist.all_gather(outs, t, group=self.group)
        return np.concatenate([o.numpy()[:counts[r]] for r, o in enumerate(outs)])

    def allreduce(self, vals: np.ndarray, op: int) -> np.ndarray:
        import torch
        t = torch.from_numpy(np.array(vals, dtype=np.float64))
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX if op == 1 else self.dist.ReduceOp.SUM,
                             group=self.group)
        return t.numpy()

    # ctypes entry points (must not raise into C)
    def _allgather(self, ctx, local, glob, bytes_per_row):
        try:
            rows = int(self.row_begin[self.rank + 1] - self.row_begin[self.rank])
            src = (C.c_uint8 * (rows * bytes_per_row)).from_address(local)
            out = self.allgather(bytes(src), int(bytes_per_row))
            C.memmove(glob, out.ctypes.data, out.nbytes)
            return 0
        except Exception:
            return -1

    def _allreduce(self, ctx, vals, n, op):
        try:
            arr = np.ctypeslib.as_array(vals, shape=(n,))
            arr[:] = self.allreduce(arr, op)
            return 0
        except Exception:
            return -1


class ShardHandle:
    """Owns an mdp_shard_t: this rank's rows of a row-sharded ELL MDP."""

    def __init__(self, ptr, S, row0, rows, A, k):
        self._p = ptr
        self.S, self.row0, self.rows, self.A, self.k = S, row0, rows, A, k

    @property
    def ptr(self):
        if self._p is None:
            raise ValueError("shard is closed")
        return self._p

    def close(self):
        if self._p is not None:
            lib().mdp_shard_destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mdp_shard_create(S: int, row0: int, col, val, g, gamma: float) -> ShardHandle:
    """col / val [A, rows, k] (global int32 columns; float32 or float64), g [A, rows] float64:
    rows [row0, row0 + rows) of an ELL MDP with S states."""
    A, rows, k = val.shape
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val)
    g = np.ascontiguousarray(g, dtype=np.float64)
    if col.shape != (A, rows, k) or g.shape != (A, rows):
        raise ValueError("col/val must be (A, rows, k) and g (A, rows)")
    h = C.c_void_p()
    _check(lib().mdp_shard_create(int(S), int(row0), int(rows), A, k, _ptr(col), _ptr(val),
                                  _dtype_code(val), _ptr(g), float(gamma), C.byref(h)),
           "mdp_shard_create")
    return ShardHandle(h, int(S), int(row0), int(rows), A, k)


def ipi_solve_sharded(h: ShardHandle, comm: ShardComm, o=None):
    """iGMRES-PI on the row-sharded MDP -> this rank's (v = T(V_K), pi, stats)."""
    o = o or opts()
    v = np.empty(h.rows, dtype=np.float64)
    pi = np.empty(h.rows, dtype=np.int32)
    st = mdp_stats()
    _check(lib().ipi_solve_sharded(h.ptr, C.byref(comm.c), C.byref(o), _ptr(v), _ptr(pi),
                                   C.byref(st)), "ipi_solve_sharded")
    return v, pi, st.as_dict()
