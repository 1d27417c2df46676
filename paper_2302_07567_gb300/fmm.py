"""Python binding of the C ABI in include/fmm.h (argument marshalling only).

Every step of the computation runs in the CUDA library; this module loads it
with ctypes, allocates the workspace as a torch tensor, passes device
pointers and the current CUDA stream, and turns status codes into
exceptions.  There is no fallback: if the library is missing, the first call
raises.

    plan = Plan(N, degree=6, leaf_size=128, eta=0.5, precision="fp32")
    E, B = plan.field(x, p, q)                      # torch, cuda, [N,3]
    dx, dp, dq = plan.adjoint(x, p, q, wE, wB)      # gradients of sum wE.E + wB.B
    E, B = FMMField.apply(x, p, q, plan)            # autograd-aware
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libfmm_gb300.so")

FMM_OK, FMM_EINVAL, FMM_ENOWORKSPACE, FMM_EOVERFLOW, FMM_ENONFINITE, FMM_ESTATE, FMM_ECUDA, FMM_EBOUNDS = range(8)
FMM_FP64, FMM_FP32 = 0, 1
FMM_RECOMPUTE, FMM_BOUNDS_CHECK, FMM_TIMING, FMM_SIZE_AWARE, FMM_TEST_POLY_KERNEL, FMM_GBAR_TERM = 1, 2, 4, 8, 16, 32
FMM_SERIAL = 64
EXPORT = dict(gbar=0, perm=1, nodes=2, bbox=3, axis=4, p2p=5, m2l=6, multipole=7, local=8)
STAGES = ["setup", "tree", "upward", "traversal", "host_wait", "m2l", "l2l", "p2p_l2p",
          "adj_l2pt_l2lt", "adj_m2lt", "adj_m2mt", "adj_near", "adj_source", "total", "adj_total", "adj_lists",
          "l2p", "p2m"]

_lib = None


class FMMError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        msg = lib().fmm_strerror(status).decode()
        if status == FMM_ECUDA:
            msg += " (" + lib().fmm_last_cuda_error().decode() + ")"
        super().__init__(f"{what}: {msg} [status {status}]")


class Stats(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("nodes", ctypes.c_int64), ("leaves", ctypes.c_int64),
                ("degree", ctypes.c_int32), ("leaf_size", ctypes.c_int32), ("kappa", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("eta", ctypes.c_double), ("gbar", ctypes.c_double),
                ("length_unit", ctypes.c_double), ("mass_unit", ctypes.c_double),
                ("p2p_pairs", ctypes.c_int64), ("m2l_pairs", ctypes.c_int64),
                ("p2p_interactions", ctypes.c_double), ("m2l_interactions", ctypes.c_double),
                ("cap_p2p", ctypes.c_int64), ("cap_m2l", ctypes.c_int64), ("cap_frontier", ctypes.c_int64),
                ("stage_ms", ctypes.c_double * 18)]


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library not built ({LIB_PATH}); run paper_2302_07567_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    P, I64, I32, D, U, SZ = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_uint, ctypes.c_size_t
    sig = {
        "fmm_plan_create": (I32, [ctypes.POINTER(P), I64, I32, I32, D, I32, U]),
        "fmm_step_graph_create": (I32, [P] * 12),
        "fmm_step_graph_launch": (I32, [P, P]),
        "fmm_step_graph_destroy": (I32, [P]),
        "fmm_copy": (I32, [P, P, SZ, P]),
        "fmm_plan_set_capacity": (I32, [P, I64, I64, I64]),
        "fmm_plan_workspace_bytes": (I32, [P, ctypes.POINTER(SZ)]),
        "fmm_plan_set_workspace": (I32, [P, P, SZ]),
        "fmm_field": (I32, [P, P, P, P, P, P, P]),
        "fmm_field_adjoint": (I32, [P, P, P, P, P, P, P, P, P, P]),
        "fmm_plan_stats": (I32, [P, ctypes.POINTER(Stats)]),
        "fmm_plan_export": (I32, [P, I32, P, SZ]),
        "fmm_direct_field": (I32, [P, P, P, I64, P, I64, D, P, P, P]),
        "fmm_plan_destroy": (None, [P]),
        "fmm_strerror": (ctypes.c_char_p, [I32]),
        "fmm_last_cuda_error": (ctypes.c_char_p, []),
        "fmm_version": (I32, []),
        "fmm_stats_bytes": (ctypes.c_size_t, []),
        "fmm_kernel_launches": (I64, []),
        "fmm_gamma_bar_noalloc": (I32, [P, I64, P, P]),
        "fmm_fp32_fma_rate": (I32, [P, SZ, I32, ctypes.POINTER(D), P]),
        "fmm_field_reuse": (I32, [P, P, P, P, P, P, P, ctypes.POINTER(I32)]),
        "fmm_boris_push": (I32, [P, P, P, I64, P, P, I32, D, D, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    if L.fmm_stats_bytes() != ctypes.sizeof(Stats):
        raise RuntimeError(f"fmm_stats layout mismatch: library {L.fmm_stats_bytes()} bytes, "
                           f"binding {ctypes.sizeof(Stats)}")
    _lib = L
    return L


def _ptr(t: torch.Tensor | None):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(device) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _check_in(t: torch.Tensor, name: str, shape, dtype, device):
    if not isinstance(t, torch.Tensor) or t.device != device or t.dtype != dtype:
        raise TypeError(f"{name} must be a {dtype} tensor on {device}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


class Plan:
    """An FMM plan (Alg. 12's FMM(S, s, N0, eta)) with its device workspace."""

    def __init__(self, N: int, degree: int, leaf_size: int, eta: float, precision: str = "fp32",
                 flags: int = 0, device=None, capacity=None):
        self.N = int(N)
        self.degree = int(degree)
        self.leaf_size = int(leaf_size)
        self.eta = float(eta)
        self.precision = precision
        self.flags = int(flags)
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.out_dtype = torch.float32 if precision == "fp32" else torch.float64
        prec = {"fp32": FMM_FP32, "fp64": FMM_FP64}[precision]
        h = ctypes.c_void_p()
        rc = lib().fmm_plan_create(ctypes.byref(h), self.N, self.degree, self.leaf_size, self.eta, prec, self.flags)
        if rc != FMM_OK:
            raise FMMError(rc, "fmm_plan_create")
        self._h = h
        self._ws = None
        self.generation = 0  # bumped by every field() call
        self.last_rebuilt = True
        if capacity is not None:
            self.set_capacity(*capacity)
        self._attach()

    # -- workspace
    def _attach(self):
        n = ctypes.c_size_t()
        rc = lib().fmm_plan_workspace_bytes(self._h, ctypes.byref(n))
        if rc != FMM_OK:
            raise FMMError(rc, "fmm_plan_workspace_bytes")
        self._ws = torch.empty(int(n.value) + 256, dtype=torch.uint8, device=self.device)
        base = self._ws.data_ptr()
        aligned = (base + 255) & ~255
        with torch.cuda.device(self.device):
            rc = lib().fmm_plan_set_workspace(self._h, ctypes.c_void_p(aligned), int(n.value))
        if rc != FMM_OK:
            raise FMMError(rc, "fmm_plan_set_workspace")

    @property
    def workspace_bytes(self) -> int:
        return 0 if self._ws is None else int(self._ws.numel())

    def set_capacity(self, p2p_pairs=0, m2l_pairs=0, frontier_pairs=0):
        rc = lib().fmm_plan_set_capacity(self._h, int(p2p_pairs), int(m2l_pairs), int(frontier_pairs))
        if rc != FMM_OK:
            raise FMMError(rc, "fmm_plan_set_capacity")
        self._ws = None
        self._attach()

    # -- compute
    def field(self, x, p, q, E=None, B=None, max_retries: int = 10, reuse: bool = False):
        """E, B [N,3] (float32 for fp32 plans, float64 for fp64) of the particles.

        On an interaction-list overflow the capacities grow (x4, or to 1.25x
        the counts seen) and the call is repeated, up to ``max_retries`` times.
        With ``reuse`` (a tracking step, fmm_field_reuse) the tree membership
        and the interaction lists of the last call stay while they remain
        admissible; ``last_rebuilt`` tells whether this call built them anew.
        """
        N, dev = self.N, self.device
        _check_in(x, "x", (N, 3), torch.float64, dev)
        _check_in(p, "p", (N, 3), torch.float64, dev)
        _check_in(q, "q", (N,), torch.float64, dev)
        if E is None:
            E = torch.empty((N, 3), dtype=self.out_dtype, device=dev)
        if B is None:
            B = torch.empty((N, 3), dtype=self.out_dtype, device=dev)
        _check_in(E, "E", (N, 3), self.out_dtype, dev)
        _check_in(B, "B", (N, 3), self.out_dtype, dev)
        rebuilt = ctypes.c_int(1)
        for _ in range(max_retries + 1):
            with torch.cuda.device(dev):
                if reuse:
                    rc = lib().fmm_field_reuse(self._h, _ptr(x), _ptr(p), _ptr(q), _ptr(E), _ptr(B), _stream(dev),
                                               ctypes.byref(rebuilt))
                else:
                    rc = lib().fmm_field(self._h, _ptr(x), _ptr(p), _ptr(q), _ptr(E), _ptr(B), _stream(dev))
            if rc != FMM_EOVERFLOW:
                break
            self._grow()
        if rc != FMM_OK:
            raise FMMError(rc, "fmm_field_reuse" if reuse else "fmm_field")
        self.generation += 1
        self.last_rebuilt = bool(rebuilt.value)
        return E, B

    def _grow(self):
        # the traversal counts every pair it finds, also past a full list: a
        # list that overflowed grows to 1.25 times its count (at least
        # doubling); with both lists within their capacities it was the
        # traversal frontier that overflowed, which grows fourfold
        st = self.stats()
        p2p_over = st["p2p_pairs"] > st["cap_p2p"]
        m2l_over = st["m2l_pairs"] > st["cap_m2l"]
        grow = lambda cap, cnt: max(2 * cap, int(1.25 * cnt) + 1024)  # noqa: E731
        self.set_capacity(grow(st["cap_p2p"], st["p2p_pairs"]) if p2p_over else 0,
                          grow(st["cap_m2l"], st["m2l_pairs"]) if m2l_over else 0,
                          0 if (p2p_over or m2l_over) else 4 * st["cap_frontier"])

    # -- recorded steps (CUDA graphs)
    def record_step(self, x, p, q, wE=None, wB=None, max_retries: int = 10):
        """Record one step, field() and with wE, wB also adjoint(), on these
        tensors as CUDA graphs (fmm_step_graph_create); returns the tensors the
        replays write: (E, B), or (E, B, dx, dp, dq) with the adjoint.

        The graphs hold the tensors' addresses: keep them (the plan keeps a
        reference) and update their contents in place between replay() calls.
        The recording runs the step once (growing the capacities on an
        overflow, as field() does) and uses a stream of the plan's own, since
        the legacy default stream cannot be recorded.
        """
        N, dev = self.N, self.device
        _check_in(x, "x", (N, 3), torch.float64, dev)
        _check_in(p, "p", (N, 3), torch.float64, dev)
        _check_in(q, "q", (N,), torch.float64, dev)
        adj = wE is not None
        if adj:
            _check_in(wE, "wE", (N, 3), self.out_dtype, dev)
            _check_in(wB, "wB", (N, 3), self.out_dtype, dev)
        E = torch.empty((N, 3), dtype=self.out_dtype, device=dev)
        B = torch.empty((N, 3), dtype=self.out_dtype, device=dev)
        grads = [torch.empty(sh, dtype=torch.float64, device=dev) for sh in ((N, 3), (N, 3), (N,))] if adj else []
        if getattr(self, "_gstream", None) is None:
            self._gstream = torch.cuda.Stream(dev)
        gs = self._gstream
        nul = ctypes.c_void_p(None)
        for _ in range(max_retries + 1):
            gs.wait_stream(torch.cuda.current_stream(dev))
            with torch.cuda.device(dev):
                rc = lib().fmm_step_graph_create(
                    self._h, _ptr(x), _ptr(p), _ptr(q), _ptr(wE) if adj else nul, _ptr(wB) if adj else nul,
                    _ptr(E), _ptr(B), *([_ptr(g) for g in grads] if adj else [nul, nul, nul]),
                    ctypes.c_void_p(gs.cuda_stream))
            if rc != FMM_EOVERFLOW:
                break
            self._grow()
        if rc != FMM_OK:
            raise FMMError(rc, "fmm_step_graph_create")
        self._graph_refs = (x, p, q, wE, wB, E, B, *grads)
        self.generation += 1
        return (E, B, *grads)

    def replay(self):
        """Replay the recorded step (fmm_step_graph_launch) after the work
        queued so far on the current stream, and wait for it.  Raises FMMError
        on an overflow (grow the capacities and record_step() again)."""
        dev = self.device
        gs = getattr(self, "_gstream", None)
        if gs is None:  # nothing recorded: the library reports FMM_ESTATE
            gs = torch.cuda.current_stream(dev)
        gs.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.device(dev):
            rc = lib().fmm_step_graph_launch(self._h, ctypes.c_void_p(gs.cuda_stream))
        if rc != FMM_OK:
            raise FMMError(rc, "fmm_step_graph_launch")
        self.generation += 1

    def adjoint(self, x, p, q, wE, wB):
        """(dL/dx, dL/dp, dL/dq) of L = sum wE.E + wB.B at the last field() call."""
        N, dev = self.N, self.device
        _check_in(wE, "wE", (N, 3), self.out_dtype, dev)
        _check_in(wB, "wB", (N, 3), self.out_dtype, dev)
        dx = torch.empty((N, 3), dtype=torch.float64, device=dev)
        dp = torch.empty((N, 3), dtype=torch.float64, device=dev)
        dq = torch.empty((N,), dtype=torch.float64, device=dev)
        with torch.cuda.device(dev):
            rc = lib().fmm_field_adjoint(self._h, _ptr(x), _ptr(p), _ptr(q), _ptr(wE), _ptr(wB), _ptr(dx),
                                         _ptr(dp), _ptr(dq), _stream(dev))
        if rc != FMM_OK:
            raise FMMError(rc, "fmm_field_adjoint")
        return dx, dp, dq

    def stats(self) -> dict:
        s = Stats()
        rc = lib().fmm_plan_stats(self._h, ctypes.byref(s))
        if rc != FMM_OK:
            raise FMMError(rc, "fmm_plan_stats")
        d = {name: getattr(s, name) for name, _ in Stats._fields_ if name != "stage_ms"}
        d["stage_ms"] = {STAGES[k]: s.stage_ms[k] for k in range(18)}
        return d

    def export(self, what: str) -> np.ndarray:
        st = self.stats()
        C, N, m = st["nodes"], st["N"], (self.degree + 1) ** 3
        shapes = dict(gbar=((1,), np.float64), perm=((N,), np.int32), nodes=((C, 2), np.int64),
                      bbox=((C, 6), np.float64), axis=((C,), np.int32), p2p=((st["p2p_pairs"], 2), np.int32),
                      m2l=((st["m2l_pairs"], 2), np.int32), multipole=((C, 4, m), np.float64),
                      local=((C, 6, m), np.float64))
        shape, dt = shapes[what]
        out = np.zeros(shape, dtype=dt)
        rc = lib().fmm_plan_export(self._h, EXPORT[what], out.ctypes.data_as(ctypes.c_void_p), out.nbytes)
        if rc != FMM_OK:
            raise FMMError(rc, f"fmm_plan_export({what})")
        return out

    def close(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.fmm_plan_destroy(self._h)
            self._h = None
        self._ws = None
        self._graph_refs = None

    def __del__(self):  # pragma: no cover - best effort
        try:
            self.close()
        except Exception:
            pass


def copy_(dst: torch.Tensor, src: torch.Tensor) -> torch.Tensor:
    """dst <- src by a kernel on the GPU's SMs (fmm_copy): a CUDA tensor and a
    pinned CPU tensor, either way, or two CUDA tensors of one device; the
    same dtype and number of elements, contiguous, 16-byte aligned, a
    multiple of 16 bytes.  Asynchronous on the CUDA tensor's current stream."""
    if dst.dtype != src.dtype or dst.numel() != src.numel():
        raise ValueError("copy_: dst and src differ in dtype or size")
    if not (dst.is_contiguous() and src.is_contiguous()):
        raise ValueError("copy_: tensors must be contiguous")
    cuda = [t for t in (dst, src) if t.is_cuda]
    if not cuda:
        raise ValueError("copy_: one tensor must be a CUDA tensor")
    for t in (dst, src):
        if not t.is_cuda and not t.is_pinned():
            raise ValueError("copy_: a CPU tensor must be pinned")
    dev = cuda[0].device
    with torch.cuda.device(dev):
        rc = lib().fmm_copy(_ptr(dst), _ptr(src), dst.numel() * dst.element_size(), _stream(dev))
    if rc != FMM_OK:
        raise FMMError(rc, "fmm_copy")
    return dst


def kernel_launches() -> int:
    """Kernels launched by the library in this process so far."""
    return int(lib().fmm_kernel_launches())


def boris_push(x, p, q, E, B, mass: float, dt: float):
    """One relativistic Boris step (fmm_boris_push): x, p updated in place."""
    dev = x.device
    N = x.shape[0]
    _check_in(x, "x", (N, 3), torch.float64, dev)
    _check_in(p, "p", (N, 3), torch.float64, dev)
    _check_in(q, "q", (N,), torch.float64, dev)
    if E.dtype not in (torch.float32, torch.float64) or B.dtype != E.dtype:
        raise TypeError("E and B must both be float32 or both float64")
    _check_in(E, "E", (N, 3), E.dtype, dev)
    _check_in(B, "B", (N, 3), E.dtype, dev)
    prec = FMM_FP32 if E.dtype == torch.float32 else FMM_FP64
    with torch.cuda.device(dev):
        rc = lib().fmm_boris_push(_ptr(x), _ptr(p), _ptr(q), N, _ptr(E), _ptr(B), prec, float(mass), float(dt),
                                  _stream(dev))
    if rc != FMM_OK:
        raise FMMError(rc, "fmm_boris_push")


def track(plan: "Plan", x, p, q, mass: float, dt: float, steps: int, reuse: bool = True) -> int:
    """Advance the beam ``steps`` time steps in its own space-charge field:
    each step the FMM field (with the previous step's tree and lists while
    they stay admissible, if ``reuse``) and a Boris push; x and p are
    updated in place.  Returns how many steps built tree and lists anew."""
    rebuilds = 0
    for _ in range(int(steps)):
        E, B = plan.field(x, p, q, reuse=reuse)
        rebuilds += int(plan.last_rebuilt) if reuse else 1
        boris_push(x, p, q, E, B, mass, dt)
    return rebuilds


def fp32_fma_rate(paired: bool, device=None) -> float:
    """Measured FP32 FMA throughput of the device in TFLOP/s (FMA = 2 flop)."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sink = torch.empty(sms * 8 * 256, dtype=torch.float32, device=dev)
    out = ctypes.c_double()
    with torch.cuda.device(dev):
        rc = lib().fmm_fp32_fma_rate(_ptr(sink), sink.numel() * 4, int(bool(paired)), ctypes.byref(out), _stream(dev))
    if rc != FMM_OK:
        raise FMMError(rc, "fmm_fp32_fma_rate")
    return float(out.value)


def direct_field(x, p, q, gbar: float, targets=None):
    """FP64 brute force (Section 5) at the rows ``targets`` (all by default)."""
    dev = x.device
    N = x.shape[0]
    _check_in(x, "x", (N, 3), torch.float64, dev)
    _check_in(p, "p", (N, 3), torch.float64, dev)
    _check_in(q, "q", (N,), torch.float64, dev)
    if targets is not None:
        targets = torch.as_tensor(targets, dtype=torch.int64, device=dev).contiguous()
        T = targets.numel()
    else:
        T = N
    E = torch.empty((T, 3), dtype=torch.float64, device=dev)
    B = torch.empty((T, 3), dtype=torch.float64, device=dev)
    with torch.cuda.device(dev):
        rc = lib().fmm_direct_field(_ptr(x), _ptr(p), _ptr(q), N, _ptr(targets), T, float(gbar), _ptr(E), _ptr(B),
                                    _stream(dev))
    if rc != FMM_OK:
        raise FMMError(rc, "fmm_direct_field")
    return E, B


class FMMField(torch.autograd.Function):
    """(E, B) = FMM(x, p, q) with the hand-written adjoint as its backward."""

    @staticmethod
    def forward(ctx, x, p, q, plan: Plan):
        E, B = plan.field(x.detach().contiguous(), p.detach().contiguous(), q.detach().contiguous())
        ctx.plan = plan
        ctx.generation = plan.generation
        ctx.save_for_backward(x, p, q)
        return E, B

    @staticmethod
    def backward(ctx, gE, gB):
        x, p, q = ctx.saved_tensors
        plan = ctx.plan
        if plan.generation != ctx.generation:  # the plan ran other inputs since: redo this forward
            plan.field(x.detach().contiguous(), p.detach().contiguous(), q.detach().contiguous())
        gE = torch.zeros((plan.N, 3), dtype=plan.out_dtype, device=plan.device) if gE is None else gE
        gB = torch.zeros((plan.N, 3), dtype=plan.out_dtype, device=plan.device) if gB is None else gB
        dx, dp, dq = plan.adjoint(x.detach().contiguous(), p.detach().contiguous(), q.detach().contiguous(),
                                  gE.to(plan.out_dtype).contiguous(), gB.to(plan.out_dtype).contiguous())
        return dx, dp, dq, None
