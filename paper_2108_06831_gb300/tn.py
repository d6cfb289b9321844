"""Thin ctypes binding of libtnq (C ABI in include/tn.h).

Argument marshalling only: every step of a contraction runs in the library's CUDA
kernels; PyTorch supplies device memory and the current stream.  The library must
have been built (``paper_2108_06831_gb300._build.build()``); importing this module
raises if ``libtnq.so`` is missing - there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

from .circuits import Circuit, PauliSum

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libtnq.so")
if not os.path.exists(_LIB_PATH):
    raise RuntimeError(f"libtnq.so is not built ({_LIB_PATH}); run paper_2108_06831_gb300._build.build()")
_lib = C.CDLL(_LIB_PATH)

OK, ERR_INVALID_ARG, ERR_UNSUPPORTED, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_NUMERIC = range(7)
TARGET_STATE, TARGET_AMPLITUDES, TARGET_EXPECTATION = 0, 1, 2
PREC_FP32, PREC_3XTF32, PREC_SPLIT_BF16 = 0, 1, 2
PLAN_HOST_ONLY = 1
PLAN_NO_SPECIALIZE = 2
PLAN_NETWORK = 4
PLAN_Q428 = 8
PLAN_NO_FUSION = 16
PLAN_BLOCKS = 32

GATE_KINDS = {name: i for i, name in enumerate(
    ["H", "X", "Y", "Z", "S", "SDG", "T", "TDG", "SX", "SY", "SW", "RX", "RY", "RZ", "U3",
     "CZ", "CNOT", "CP", "SWAP", "MAT1", "MAT2"])}
PAULI_CODE = {"I": 0, "X": 1, "Y": 2, "Z": 3}


class TnGate(C.Structure):
    _fields_ = [("kind", C.c_int32), ("q", C.c_int32 * 2), ("param_idx", C.c_int32),
                ("angle", C.c_double * 3), ("mat", C.POINTER(C.c_double))]


class TnPlanOpts(C.Structure):
    _fields_ = [("target", C.c_int32), ("precision", C.c_int32), ("batch", C.c_int32),
                ("tile_qubits", C.c_int32), ("max_intermediate_log2", C.c_int32), ("flags", C.c_int32),
                ("seed", C.c_uint64), ("amp_batch", C.c_int64), ("order_trials", C.c_int64),
                ("order_search", C.c_int64), ("block_qubits", C.c_int64),
                ("reserved", C.c_int64 * 2)]


class TnPlanStats(C.Structure):
    _fields_ = [("n_qubits", C.c_int32), ("n_params", C.c_int32), ("n_gates", C.c_int64),
                ("n_passes", C.c_int32), ("n_phases", C.c_int32), ("n_ops", C.c_int64),
                ("tile_qubits", C.c_int32), ("reg_qubits", C.c_int32), ("hbm_bytes", C.c_double),
                ("flops", C.c_double), ("n_bwd_passes", C.c_int32), ("specialized", C.c_int32),
                ("net_merges", C.c_int32), ("net_max_log2", C.c_int32), ("net_tensor_merges", C.c_int32),
                ("net_folded_merges", C.c_int32), ("bwd_flops", C.c_double),
                ("net_sliced", C.c_int32), ("net_batch_log2", C.c_int32), ("net_cost", C.c_double),
                ("net_bytes", C.c_double), ("n_fused", C.c_int32), ("reserved_stats", C.c_int32)]


class TnTuneOpts(C.Structure):
    _fields_ = [("candidates", C.c_int32 * 8), ("reps", C.c_int32), ("flags", C.c_int32),
                ("reserved", C.c_int64 * 4)]


class TnPauliSum(C.Structure):
    _fields_ = [("n_terms", C.c_int32), ("coef", C.POINTER(C.c_double)), ("paulis", C.POINTER(C.c_uint8))]


_vp = C.c_void_p
_sigs = {
    "tn_build_from_circuit": [C.c_int32, C.POINTER(TnGate), C.c_int64, C.c_uint64, C.POINTER(_vp)],
    "tn_circuit_num_params": [_vp, C.POINTER(C.c_int32)],
    "tn_free_circuit": [_vp],
    "tn_plan_contraction": [_vp, C.POINTER(TnPlanOpts), C.POINTER(_vp)],
    "tn_plan_workspace_bytes": [_vp, C.POINTER(C.c_size_t)],
    "tn_plan_get_stats": [_vp, C.POINTER(TnPlanStats)],
    "tn_free_plan": [_vp],
    "tn_build_observable": [C.c_int32, C.POINTER(TnPauliSum), C.POINTER(_vp)],
    "tn_free_observable": [_vp],
    "tn_contract_state": [_vp, _vp, _vp, _vp, _vp],
    "tn_contract_state_q428": [_vp, _vp, _vp],
    "tn_contract_amplitudes": [_vp, _vp, _vp, C.c_int64, _vp, _vp, _vp],
    "tn_expectation": [_vp, _vp, _vp, _vp, _vp, _vp],
    "tn_expectation_backward": [_vp, _vp, _vp, _vp, _vp, _vp, _vp],
    "tn_expectation_value_and_grad": [_vp, _vp, _vp, _vp, _vp, _vp, _vp],
    "tn_state_expectation_workspace_bytes": [_vp, C.c_int32, C.POINTER(C.c_size_t)],
    "tn_state_expectation": [_vp, C.c_int32, _vp, _vp, _vp, C.c_size_t, _vp],
    "tn_state_expectation_noalloc": [_vp, C.c_int32, _vp, _vp, _vp],
    "tn_permute": [C.c_int32, C.POINTER(C.c_int32), C.c_int64, _vp, _vp, _vp],
    "tn_cgemm_workspace_bytes": [C.c_int32, C.c_int64, C.c_int64, C.c_int64, C.c_int64, C.POINTER(C.c_size_t)],
    "tn_cgemm_batched": [C.c_int32, C.c_int64, C.c_int64, C.c_int64, C.c_int64, _vp, _vp, _vp, _vp, C.c_size_t, _vp],
    "tn_batch_build": [C.POINTER(_vp), C.c_int32, C.POINTER(_vp)],
    "tn_batch_sizes": [_vp, C.POINTER(C.c_int64), C.POINTER(C.c_size_t)],
    "tn_batch_state_offsets": [_vp, C.POINTER(C.c_int64)],
    "tn_batch_run": [_vp, _vp, _vp, _vp],
    "tn_free_batch": [_vp],
    "tn_batch_test_stall": [_vp, C.c_int32, C.c_int32, C.c_int64],
    "tn_batch_run_params": [_vp, _vp, _vp, _vp, _vp],
    "tn_plan_contraction_tuned": [_vp, C.POINTER(TnPlanOpts), C.POINTER(TnTuneOpts), _vp, C.POINTER(_vp),
                                  C.POINTER(C.c_int32)],
    "tn_batch_params": [_vp, C.POINTER(C.c_int32), C.POINTER(C.c_int64)],
    "tn_probe_fma_rate": [C.POINTER(C.c_double), C.POINTER(C.c_double)],
    "tn_batch_build_tuned": [C.POINTER(_vp), C.c_int32, C.POINTER(TnTuneOpts), _vp, C.POINTER(_vp),
                             C.POINTER(C.c_int32)],
    "tn_sync_status": [_vp],
    "tn_last_error": [],
    "tn_version": [],
}
for _name, _args in _sigs.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = None if _name.startswith("tn_free") else (C.c_char_p if _name in ("tn_last_error", "tn_version") else C.c_int)

EXPORTED = tuple(_sigs)


class TnError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = _lib.tn_last_error().decode(errors="replace")
        super().__init__(f"{where} failed with status {status}: {msg}")


def _check(status: int, where: str) -> None:
    if status != OK:
        raise TnError(status, where)


def version() -> str:
    return _lib.tn_version().decode()


def _ptr(t) -> Optional[int]:
    """Device (or host) address of a tensor/array, None for None."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return int(t)


def _stream(stream) -> Optional[int]:
    if stream is not None:
        return int(stream) if isinstance(stream, int) else stream.cuda_stream
    import torch
    return torch.cuda.current_stream().cuda_stream


# ----------------------------------------------------------------------------- handles

class CircuitHandle:
    def __init__(self, circ: Circuit):
        n = len(circ.gates)
        arr = (TnGate * max(n, 1))()
        self._mats = []
        for i, g in enumerate(circ.gates):
            t = arr[i]
            t.kind = GATE_KINDS[g.kind]
            t.q[0] = g.qubits[0]
            t.q[1] = g.qubits[1] if len(g.qubits) > 1 else 0
            t.param_idx = g.param_idx
            for a, v in enumerate(g.angles[:3]):
                t.angle[a] = v
            if g.mat is not None:
                m = np.empty(2 * len(g.mat), dtype=np.float64)
                m[0::2] = [complex(z).real for z in g.mat]
                m[1::2] = [complex(z).imag for z in g.mat]
                self._mats.append(m)
                t.mat = m.ctypes.data_as(C.POINTER(C.c_double))
        h = _vp()
        _check(_lib.tn_build_from_circuit(circ.n_qubits, arr, n, circ.init_basis, C.byref(h)), "tn_build_from_circuit")
        self._h = h
        self.n_qubits = circ.n_qubits
        np_ = C.c_int32()
        _check(_lib.tn_circuit_num_params(h, C.byref(np_)), "tn_circuit_num_params")
        self.n_params = np_.value

    def __del__(self):
        if getattr(self, "_h", None):
            _lib.tn_free_circuit(self._h)
            self._h = None


class Plan:
    def __init__(self, ch: CircuitHandle, target: int = TARGET_STATE, precision: int = PREC_FP32, batch: int = 1,
                 tile_qubits: int = 0, host_only: bool = False, specialize: bool = True, network_bitstrings: int = 0,
                 max_intermediate_log2: int = 0, order_trials: int = 0, q428: bool = False, order_search: int = 0,
                 fuse: bool = True, block_qubits: int = 0, tune: Optional[dict] = None):
        o = TnPlanOpts()
        o.order_trials = order_trials
        o.order_search = order_search
        o.target, o.precision, o.batch, o.tile_qubits = target, precision, batch, tile_qubits
        o.max_intermediate_log2 = max_intermediate_log2
        o.flags = (PLAN_HOST_ONLY if host_only else 0) | (0 if specialize else PLAN_NO_SPECIALIZE) | \
            (PLAN_Q428 if q428 else 0) | (0 if fuse else PLAN_NO_FUSION) | (PLAN_BLOCKS if block_qubits else 0)
        o.block_qubits = block_qubits
        if network_bitstrings:
            o.flags |= PLAN_NETWORK
            o.amp_batch = network_bitstrings
        h = _vp()
        self.tuned_tile = None
        if tune is not None:  # tile size picked by measurement (tn_plan_contraction_tuned)
            t = TnTuneOpts()
            for i, cnd in enumerate(list(tune.get("candidates", ()))[:8]):
                t.candidates[i] = int(cnd)
            t.reps = int(tune.get("reps", 0))
            tile = C.c_int32()
            _check(_lib.tn_plan_contraction_tuned(ch._h, C.byref(o), C.byref(t), _stream(tune.get("stream")),
                                                  C.byref(h), C.byref(tile)), "tn_plan_contraction_tuned")
            self.tuned_tile = tile.value
        else:
            _check(_lib.tn_plan_contraction(ch._h, C.byref(o), C.byref(h)), "tn_plan_contraction")
        self._h = h
        self.circuit = ch
        self.n_qubits, self.n_params, self.batch, self.target = ch.n_qubits, ch.n_params, batch, target
        ws = C.c_size_t()
        _check(_lib.tn_plan_workspace_bytes(h, C.byref(ws)), "tn_plan_workspace_bytes")
        self.workspace_bytes = ws.value

    def stats(self) -> dict:
        s = TnPlanStats()
        _check(_lib.tn_plan_get_stats(self._h, C.byref(s)), "tn_plan_get_stats")
        return {f: getattr(s, f) for f, _ in TnPlanStats._fields_ if not f.startswith("reserved")}

    def __del__(self):
        if getattr(self, "_h", None):
            _lib.tn_free_plan(self._h)
            self._h = None


class Observable:
    def __init__(self, H: PauliSum):
        coef = np.asarray(H.coef, dtype=np.float64)
        codes = np.array([[PAULI_CODE[p] for p in s] for s in H.strings], dtype=np.uint8).reshape(-1)
        ps = TnPauliSum()
        ps.n_terms = len(H.coef)
        ps.coef = coef.ctypes.data_as(C.POINTER(C.c_double))
        ps.paulis = codes.ctypes.data_as(C.POINTER(C.c_uint8))
        h = _vp()
        _check(_lib.tn_build_observable(H.n_qubits, C.byref(ps), C.byref(h)), "tn_build_observable")
        self._h = h
        self.n_qubits = H.n_qubits

    def __del__(self):
        if getattr(self, "_h", None):
            _lib.tn_free_observable(self._h)
            self._h = None


# ----------------------------------------------------------------------------- calls (same names as the C ABI)

def build_from_circuit(circ: Circuit) -> CircuitHandle:
    return CircuitHandle(circ)


def plan_contraction(ch: CircuitHandle, **kw) -> Plan:
    return Plan(ch, **kw)


def build_observable(H: PauliSum) -> Observable:
    return Observable(H)


def contract_state(plan: Plan, params, state, workspace, stream=None) -> None:
    _check(_lib.tn_contract_state(plan._h, _ptr(params), _ptr(state), _ptr(workspace), _stream(stream)),
           "tn_contract_state")


def contract_state_q428(plan: Plan, state, stream=None) -> None:
    """Fixed-point (Q4.28) contraction of a plan built with q428=True; state: int32 [2^N, 2] on the device."""
    _check(_lib.tn_contract_state_q428(plan._h, _ptr(state), _stream(stream)), "tn_contract_state_q428")


def contract_amplitudes(plan: Plan, params, bitstrings, amps, workspace, stream=None) -> None:
    n = 0 if bitstrings is None else int(bitstrings.numel())
    _check(_lib.tn_contract_amplitudes(plan._h, _ptr(params), _ptr(bitstrings), n, _ptr(amps), _ptr(workspace),
                                       _stream(stream)), "tn_contract_amplitudes")


def expectation(plan: Plan, obs: Observable, params, out, workspace, stream=None) -> None:
    _check(_lib.tn_expectation(plan._h, obs._h, _ptr(params), _ptr(out), _ptr(workspace), _stream(stream)),
           "tn_expectation")


def expectation_backward(plan: Plan, obs: Observable, params, grad_out, grad_params, workspace, stream=None) -> None:
    _check(_lib.tn_expectation_backward(plan._h, obs._h, _ptr(params), _ptr(grad_out), _ptr(grad_params),
                                        _ptr(workspace), _stream(stream)), "tn_expectation_backward")


def expectation_value_and_grad(plan: Plan, obs: Observable, params, out, grad_params, workspace, stream=None) -> None:
    _check(_lib.tn_expectation_value_and_grad(plan._h, obs._h, _ptr(params), _ptr(out), _ptr(grad_params),
                                              _ptr(workspace), _stream(stream)), "tn_expectation_value_and_grad")


def state_expectation_workspace_bytes(obs: Observable, batch: int) -> int:
    b = C.c_size_t()
    _check(_lib.tn_state_expectation_workspace_bytes(obs._h, batch, C.byref(b)), "tn_state_expectation_workspace_bytes")
    return b.value


def state_expectation(obs: Observable, batch: int, state, out, workspace, workspace_bytes: int, stream=None) -> None:
    _check(_lib.tn_state_expectation(obs._h, batch, _ptr(state), _ptr(out), _ptr(workspace), workspace_bytes,
                                     _stream(stream)), "tn_state_expectation")


def state_expectation_noalloc(obs: Observable, batch: int, state, out, stream=None) -> None:
    """tn_state_expectation without a workspace (scratch compiled into the library)."""
    _check(_lib.tn_state_expectation_noalloc(obs._h, batch, _ptr(state), _ptr(out), _stream(stream)),
           "tn_state_expectation_noalloc")


def permute(n_legs: int, perm: Sequence[int], batch: int, inp, out, stream=None) -> None:
    p = (C.c_int32 * n_legs)(*perm)
    _check(_lib.tn_permute(n_legs, p, batch, _ptr(inp), _ptr(out), _stream(stream)), "tn_permute")


def cgemm_workspace_bytes(precision: int, batch: int, M: int, N: int, K: int) -> int:
    b = C.c_size_t()
    _check(_lib.tn_cgemm_workspace_bytes(precision, batch, M, N, K, C.byref(b)), "tn_cgemm_workspace_bytes")
    return b.value


def cgemm_batched(precision: int, batch: int, M: int, N: int, K: int, A, B, Cm, workspace=None, workspace_bytes: int = 0,
                  stream=None) -> None:
    _check(_lib.tn_cgemm_batched(precision, batch, M, N, K, _ptr(A), _ptr(B), _ptr(Cm), _ptr(workspace),
                                 workspace_bytes, _stream(stream)), "tn_cgemm_batched")


class Batch:
    """Many circuits (fixed angles, or parameters read per run) contracted by one persistent launch
    (tn_batch_*); circuits of 19 qubits and more whose plans carry generated kernels run those on
    the batch's side streams beside it."""

    def __init__(self, plans: Sequence[Plan]):
        arr = (_vp * len(plans))(*[p._h for p in plans])
        h = _vp()
        _check(_lib.tn_batch_build(arr, len(plans), C.byref(h)), "tn_batch_build")
        self.plans = list(plans)
        self.tiles = [p.stats()["tile_qubits"] for p in plans]
        self._init(h, len(plans))

    @classmethod
    def tuned(cls, circuits: Sequence["CircuitHandle"], candidates: Sequence[int] = (), reps: int = 3,
              stream=None) -> "Batch":
        """Batch whose tile sizes are picked by measurement (tn_batch_build_tuned); it owns its plans."""
        o = TnTuneOpts()
        for i, c in enumerate(list(candidates)[:8]):
            o.candidates[i] = int(c)
        o.reps = reps
        arr = (_vp * len(circuits))(*[c._h for c in circuits])
        tiles = (C.c_int32 * len(circuits))()
        h = _vp()
        _check(_lib.tn_batch_build_tuned(arr, len(circuits), C.byref(o), _stream(stream), C.byref(h), tiles),
               "tn_batch_build_tuned")
        self = cls.__new__(cls)
        self.plans = []
        self.circuits = list(circuits)
        self.tiles = list(tiles)
        self._init(h, len(circuits))
        return self

    def _init(self, h, n):
        self._h = h
        e = C.c_int64()
        w = C.c_size_t()
        _check(_lib.tn_batch_sizes(h, C.byref(e), C.byref(w)), "tn_batch_sizes")
        self.state_elems, self.workspace_bytes = e.value, w.value
        offs = (C.c_int64 * n)()
        _check(_lib.tn_batch_state_offsets(h, offs), "tn_batch_state_offsets")
        self.offsets = list(offs)
        npar = C.c_int32()
        poffs = (C.c_int64 * n)()
        _check(_lib.tn_batch_params(h, C.byref(npar), poffs), "tn_batch_params")
        self.n_params, self.param_offsets = npar.value, list(poffs)

    def __del__(self):
        if getattr(self, "_h", None):
            _lib.tn_free_batch(self._h)
            self._h = None


def batch_run(batch: Batch, states, workspace, stream=None, params=None) -> None:
    """One persistent launch over every circuit of the batch; params (device float64, all circuits'
    parameters back to back at batch.param_offsets) for batches with parameterised circuits."""
    if params is None:
        _check(_lib.tn_batch_run(batch._h, _ptr(states), _ptr(workspace), _stream(stream)), "tn_batch_run")
    else:
        _check(_lib.tn_batch_run_params(batch._h, _ptr(params), _ptr(states), _ptr(workspace), _stream(stream)),
               "tn_batch_run_params")


def batch_test_stall(batch: Batch, circ: int, pass_index: int = 1, wait_limit_ns: int = 0) -> None:
    """Failure-path testing aid (tn_batch_test_stall): the next runs stop at a dependency wait
    that can never be met, after wait_limit_ns; circ = -1 restores the batch."""
    _check(_lib.tn_batch_test_stall(batch._h, int(circ), int(pass_index), int(wait_limit_ns)),
           "tn_batch_test_stall")


def probe_fma_rate() -> tuple:
    """(TFLOP/s, seconds): the measured FP32 multiply-add rate of the current device."""
    r, t = C.c_double(), C.c_double()
    _check(_lib.tn_probe_fma_rate(C.byref(r), C.byref(t)), "tn_probe_fma_rate")
    return r.value, t.value


def sync_status(stream=None) -> int:
    return _lib.tn_sync_status(_stream(stream))


# ----------------------------------------------------------------------------- torch conveniences

def _torch():
    import torch
    return torch


class Contractor:
    """Plan + workspace for repeated contractions of one circuit (device memory from torch)."""

    def __init__(self, circ: Circuit, target: int = TARGET_STATE, batch: int = 1, tile_qubits: int = 0,
                 precision: int = PREC_FP32, device=None, specialize: bool = True, fuse: bool = True,
                 block_qubits: int = 0, tune: Optional[dict] = None):
        torch = _torch()
        self.device = torch.device(device or "cuda")
        with torch.cuda.device(self.device):
            self.circuit_handle = CircuitHandle(circ)
            self.plan = Plan(self.circuit_handle, target=target, precision=precision, batch=batch,
                             tile_qubits=tile_qubits, specialize=specialize, fuse=fuse,
                             block_qubits=block_qubits, tune=tune)
        self.n_qubits, self.batch, self.n_params = circ.n_qubits, batch, self.plan.n_params
        nb = max(self.plan.workspace_bytes, 16)
        self.workspace = torch.empty(nb, dtype=torch.uint8, device=self.device)

    def state(self, params=None, out=None):
        torch = _torch()
        if out is None:
            out = torch.empty((self.batch, 1 << self.n_qubits), dtype=torch.complex64, device=self.device)
        contract_state(self.plan, params, out, self.workspace)
        return out

    def amplitudes(self, bitstrings, params=None, out=None):
        torch = _torch()
        if out is None:
            out = torch.empty((self.batch, bitstrings.numel()), dtype=torch.complex64, device=self.device)
        contract_amplitudes(self.plan, params, bitstrings, out, self.workspace)
        return out

    def expectation(self, obs: Observable, params=None, out=None):
        torch = _torch()
        if out is None:
            out = torch.empty(self.batch, dtype=torch.float64, device=self.device)
        expectation(self.plan, obs, params, out, self.workspace)
        return out

    def expectation_backward(self, obs: Observable, params, grad_out=None, out=None):
        torch = _torch()
        if out is None:
            out = torch.empty((self.batch, self.n_params), dtype=torch.float64, device=self.device)
        expectation_backward(self.plan, obs, params, grad_out, out, self.workspace)
        return out

    def expectation_value_and_grad(self, obs: Observable, params):
        """(energies [batch], gradients [batch][n_params]) with one forward contraction."""
        torch = _torch()
        e = torch.empty(self.batch, dtype=torch.float64, device=self.device)
        g = torch.empty((self.batch, self.n_params), dtype=torch.float64, device=self.device)
        expectation_value_and_grad(self.plan, obs, params, e, g, self.workspace)
        return e, g


def _make_expectation_fn():
    torch = _torch()

    class ExpectationFn(torch.autograd.Function):
        """<H>(theta) with the adjoint-sweep gradient (both through libtnq)."""

        @staticmethod
        def forward(ctx, params, contractor: Contractor, obs: Observable):
            p = params.detach().to(torch.float64).contiguous()
            out = contractor.expectation(obs, p)
            ctx.save_for_backward(p)
            ctx.contractor, ctx.obs = contractor, obs
            return out

        @staticmethod
        def backward(ctx, grad_out):
            (p,) = ctx.saved_tensors
            g = ctx.contractor.expectation_backward(ctx.obs, p, grad_out.detach().to(torch.float64).contiguous())
            return g.to(p.dtype), None, None

    return ExpectationFn


_EXPECTATION_FN = None


def expectation_autograd(params, contractor: Contractor, obs: Observable):
    global _EXPECTATION_FN
    if _EXPECTATION_FN is None:
        _EXPECTATION_FN = _make_expectation_fn()
    return _EXPECTATION_FN.apply(params, contractor, obs)
