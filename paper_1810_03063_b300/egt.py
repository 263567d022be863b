"""Thin ctypes binding of libegt (include/egt.h): argument marshalling only.

Every computation runs in the CUDA library.  Device buffers are anything
with a ``data_ptr()`` (torch tensors) or a raw integer address; streams are a
``torch.cuda.Stream`` or a raw ``cudaStream_t`` integer (None = the current
torch stream when torch is loaded, else the legacy default stream).

Importing this module loads ``libegt.so`` and raises ImportError if it has not
been built (``python -m paper_1810_03063_b300.build``): there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libegt.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "egt.h")
if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_1810_03063_b300.build`")
lib = C.CDLL(LIB_PATH)

STATUS = {0: "EGT_OK", 1: "EGT_ERR_INVALID_ARG", 2: "EGT_ERR_OOM", 3: "EGT_ERR_CUDA",
          4: "EGT_ERR_NUMERIC", 5: "EGT_ERR_TAU_UNDERFLOW", 6: "EGT_ERR_NOT_CONVERGED",
          7: "EGT_ERR_TIMEOUT"}
THEORY, PRACTICAL, EGT_AS = 0, 1, 2
STEP_PLAIN, STEP_CHECK, STEP_DECR = 0, 1, 2


class EGTError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def write_log_jsonl(path, log):
    """One JSON object per accepted iteration of a solve's log (solve(..., log_cap=n)["log"]):
    t, player, tau, mu_x, mu_y, EGV, the residual before the iteration's update (mbb per hand),
    back-offs, gradient products so far (3 per Step attempt) and seconds since the first logged
    iteration."""
    import json
    products = 0
    t0 = log[0]["time_ns"] if log else 0
    with open(path, "w") as f:
        for e in log:
            products += 3 * (1 + e["backoffs"])
            rec = dict(t=e["t"], player=e["player"], tau=e["tau"], mu_x=e["mu"][0], mu_y=e["mu"][1],
                       egv=None if e["egv"] != e["egv"] else e["egv"],
                       gap_mbb=None if e["gap_mbb"] != e["gap_mbb"] else e["gap_mbb"],
                       backoffs=e["backoffs"], products=products, seconds=(e["time_ns"] - t0) * 1e-9)
            f.write(json.dumps(rec) + "\n")


class Menu(C.Structure):
    _fields_ = [("n", C.c_int32), ("fracs", C.POINTER(C.c_double)), ("allin", C.c_int32),
                ("fold", C.c_int32)]


class GameDesc(C.Structure):
    _fields_ = [("n_cards", C.c_int32), ("hand_size", C.c_int32), ("n_hands", C.c_int32),
                ("hand_cards", C.POINTER(C.c_int32)), ("strength", C.POINTER(C.c_int32)),
                ("range", C.POINTER(C.c_double) * 2), ("pot", C.c_double), ("stack", C.c_double),
                ("bb", C.c_double), ("n_bets", C.c_int32), ("bet_fracs", C.POINTER(C.c_double)),
                ("allin", C.c_int32), ("raise_cap", C.c_int32), ("menus", C.POINTER(Menu))]


class Dims(C.Structure):
    _fields_ = [("H", C.c_int32), ("ld", C.c_int32), ("S", C.c_int32 * 2), ("J", C.c_int32 * 2),
                ("L", C.c_int32 * 2), ("T", C.c_int32), ("n_fold", C.c_int32), ("Z", C.c_double),
                ("normA", C.c_double), ("M", C.c_double * 2), ("Omega", C.c_double * 2),
                ("table_bytes", C.c_int64), ("device_bytes", C.c_int64)]


class IterLog(C.Structure):
    _fields_ = [("t", C.c_int32), ("player", C.c_int32), ("backoffs", C.c_int32),
                ("tau", C.c_double), ("mu", C.c_double * 2), ("egv", C.c_double),
                ("gap_mbb", C.c_double), ("time_ns", C.c_uint64)]


class SolveOpts(C.Structure):
    _fields_ = [("variant", C.c_int32), ("alpha", C.c_double), ("mu0", C.c_double * 2),
                ("eps_mbb", C.c_double), ("max_iters", C.c_int32), ("gap_every", C.c_int32),
                ("replay_n", C.c_int32), ("replay_player", C.POINTER(C.c_int32)),
                ("replay_tau", C.POINTER(C.c_double)), ("log_cap", C.c_int32),
                ("log", C.POINTER(IterLog)), ("engine", C.c_int32)]


class SolveReport(C.Structure):
    _fields_ = [("iters", C.c_int32), ("products", C.c_int32), ("backoffs", C.c_int32),
                ("gap_checks", C.c_int32), ("gap_mbb", C.c_double), ("mu", C.c_double * 2),
                ("tau", C.c_double), ("seconds", C.c_double)]


class BatchMemberInfo(C.Structure):
    _fields_ = [("active", C.c_int32), ("status", C.c_int32), ("rep", SolveReport)]


class Checkpoint(C.Structure):
    _fields_ = [("t", C.c_int32), ("tau", C.c_double), ("mu", C.c_double * 2), ("gap_mbb", C.c_double)]


class LaunchShape(C.Structure):
    _fields_ = [("share", C.c_int32), ("pairs", C.c_int32), ("grid_pct", C.c_int32), ("pack", C.c_int32),
                ("wave_mb", C.c_int32), ("wave_min", C.c_int32)]


TUNE_MAX = 16


class TuneReport(C.Structure):
    _fields_ = [("n", C.c_int32), ("best", C.c_int32), ("shape", LaunchShape * TUNE_MAX),
                ("us_per_iter", C.c_double * TUNE_MAX), ("iters", C.c_int32 * TUNE_MAX)]


class ServerOpts(C.Structure):
    _fields_ = [("mem_budget_bytes", C.c_int64), ("max_running", C.c_int32),
                ("iters_per_step", C.c_int32), ("group", C.c_int32)]


class ServerStats(C.Structure):
    _fields_ = [("queued", C.c_int32), ("running", C.c_int32), ("completed", C.c_int64),
                ("launches", C.c_int64), ("used_bytes", C.c_int64), ("budget_bytes", C.c_int64),
                ("clock", C.c_double)]


class ServerRequestInfo(C.Structure):
    _fields_ = [("state", C.c_int32), ("status", C.c_int32), ("t_submit", C.c_double),
                ("t_admit", C.c_double), ("t_done", C.c_double), ("rep", SolveReport),
                ("S", C.c_int32 * 2), ("ld", C.c_int32)]


class StepInfo(C.Structure):
    _fields_ = [("player", C.c_int32), ("accepted", C.c_int32), ("backoffs", C.c_int32),
                ("products", C.c_int32), ("tau", C.c_double), ("egv", C.c_double),
                ("mu", C.c_double * 2)]


_vp, _i32, _f64 = C.c_void_p, C.c_int32, C.c_double
_SIGS = {
    "egt_create_game": [C.POINTER(GameDesc), _i32, _vp, C.POINTER(_vp)],
    "egt_destroy_game": [_vp],
    "egt_dims_query": [_vp, C.POINTER(Dims)],
    "egt_hand_order": [_vp, _vp],
    "egt_treeplex_query": [_vp, _i32, _vp, _vp, _vp, _vp, _vp],
    "egt_terminal_query": [_vp, _vp, _vp, _vp, _vp],
    "egt_grad": [_vp, _i32, _vp, _vp, _vp],
    "egt_grad_f64": [_vp, _i32, _vp, _vp, _vp],
    "egt_smoothed_br": [_vp, _i32, _vp, _f64, _vp, C.POINTER(_f64), _vp],
    "egt_best_response_f64": [_vp, _i32, _vp, C.POINTER(_f64), _vp],
    "egt_gap": [_vp, _vp, _vp, C.POINTER(_f64), _vp],
    "egt_solver_init": [_vp, C.POINTER(SolveOpts), _vp],
    "egt_step": [_vp, _i32, C.POINTER(_f64), _i32, C.POINTER(StepInfo), _vp],
    "egt_step_point": [_vp, _vp, C.POINTER(_i32), _vp],
    "egt_state_get": [_vp, _vp, _vp, _vp, _vp],
    "egt_state_set": [_vp, _vp, _vp, _vp, _vp],
    "egt_checkpoint_get": [_vp, _vp, _vp, C.POINTER(Checkpoint), _vp],
    "egt_checkpoint_set": [_vp, _vp, _vp, C.POINTER(Checkpoint), _vp],
    "egt_solve": [_vp, C.POINTER(SolveOpts), _vp, _vp, C.POINTER(SolveReport), _vp],
    "egt_state_gap": [_vp, C.POINTER(_f64), _vp],
    "egt_gap_noalloc": [_vp, _vp, _vp, C.POINTER(_f64), _vp],
    "egt_iterate": [_vp, C.POINTER(SolveOpts), _i32, C.POINTER(SolveReport), _vp],
    "egt_engine_trace": [_vp, _i32, _vp, _vp, _vp],
    "egt_profile": [_vp, _i32],
    "egt_batch_create": [_i32, C.POINTER(_vp)],
    "egt_batch_destroy": [_vp],
    "egt_batch_add": [_vp, _vp, C.POINTER(SolveOpts), C.POINTER(_i32)],
    "egt_batch_remove": [_vp, _i32],
    "egt_batch_step": [_vp, _i32, _i32, C.POINTER(_i32), _vp],
    "egt_batch_member": [_vp, _i32, C.POINTER(BatchMemberInfo)],
    "egt_batch_launch_shape": [_vp, C.POINTER(_i32), C.POINTER(_i32)],
    "egt_batch_set_shape": [_vp, C.POINTER(LaunchShape)],
    "egt_batch_get_shape": [_vp, C.POINTER(LaunchShape)],
    "egt_batch_tune": [_vp, _i32, _i32, C.POINTER(TuneReport), _vp],
    "egt_server_create": [_i32, C.POINTER(ServerOpts), C.POINTER(_vp)],
    "egt_server_destroy": [_vp],
    "egt_server_submit": [_vp, C.POINTER(GameDesc), C.POINTER(SolveOpts), _f64, C.POINTER(C.c_int64)],
    "egt_server_step": [_vp, C.POINTER(ServerStats), _vp],
    "egt_server_result": [_vp, C.c_int64, C.POINTER(ServerRequestInfo), _vp, _vp, _i32],
    "egt_profile_read": [_vp, _vp, _vp],
}
KERNEL_KINDS = ("grad_f32", "grad_f64", "sbr", "br_f64", "engine")
ENGINE_DEVICE, ENGINE_HOST = 0, 1
for _name, _args in _SIGS.items():
    _fn = getattr(lib, _name)
    _fn.argtypes = _args
    _fn.restype = C.c_int
lib.egt_last_error.argtypes = []
lib.egt_last_error.restype = C.c_char_p
lib.egt_server_clock.argtypes = [_vp]
lib.egt_server_clock.restype = C.c_double
lib.egt_server_state_name.argtypes = [_i32]
lib.egt_server_state_name.restype = C.c_char_p


def declared_symbols(header=HEADER):
    """Names of the functions include/egt.h declares."""
    text = open(header).read()
    return sorted(set(re.findall(r"\b(egt_[a-z0-9_]+)\s*\(", text)))


def _check(status):
    if status != 0:
        raise EGTError(status, lib.egt_last_error().decode())


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(s):
    if s is None:
        import sys
        torch = sys.modules.get("torch")
        if torch is not None and torch.cuda.is_available() and torch.cuda.is_initialized():
            return torch.cuda.current_stream().cuda_stream
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _i32p(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def _f64p(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _desc(spec):
    """egt_game_desc of a synth.GameSpec, with the arrays it points into (keep them alive)."""
    keep = dict(
        cards=np.ascontiguousarray(spec.hands, dtype=np.int32),
        strength=np.ascontiguousarray(spec.strength, dtype=np.int32),
        r0=np.ascontiguousarray(spec.ranges[0], dtype=np.float64),
        r1=np.ascontiguousarray(spec.ranges[1], dtype=np.float64),
        bets=np.ascontiguousarray(spec.bet_fracs, dtype=np.float64),
    )
    d = GameDesc()
    d.n_cards = spec.n_cards
    d.hand_size = spec.hand_size
    d.n_hands = spec.n_hands
    d.hand_cards = _i32p(keep["cards"])
    d.strength = _i32p(keep["strength"])
    d.range[0] = _f64p(keep["r0"])
    d.range[1] = _f64p(keep["r1"])
    d.pot, d.stack, d.bb = spec.pot, spec.stack, spec.bb
    d.n_bets = len(spec.bet_fracs)
    d.bet_fracs = _f64p(keep["bets"])
    d.allin = int(spec.allin)
    d.raise_cap = spec.raise_cap
    menus = getattr(spec, "menus", None)
    if menus is not None:
        arr = (Menu * 8)()
        for p in range(2):
            for k in range(4):
                fr, allin, fold = menus[p][k]
                a = np.ascontiguousarray(fr, dtype=np.float64)
                keep[f"menu{p}{k}"] = a
                arr[4 * p + k] = Menu(len(fr), _f64p(a) if len(fr) else None, int(allin), int(fold))
        keep["menus"] = arr
        d.menus = C.cast(arr, C.POINTER(Menu))
    return d, keep


class Game:
    """One compiled river endgame on a device (owns its device memory)."""

    def __init__(self, spec, device=0, stream=None):
        d, self._keep = _desc(spec)
        self._h = _vp()
        _check(lib.egt_create_game(C.byref(d), device, _stream(stream), C.byref(self._h)))
        self.spec = spec
        self.device = device
        dims = Dims()
        _check(lib.egt_dims_query(self._h, C.byref(dims)))
        self.H, self.ld = dims.H, dims.ld
        self.S = (dims.S[0], dims.S[1])
        self.J = (dims.J[0], dims.J[1])
        self.L = (dims.L[0], dims.L[1])
        self.T, self.n_fold = dims.T, dims.n_fold
        self.Z, self.normA = dims.Z, dims.normA
        self.M = (dims.M[0], dims.M[1])
        self.Omega = (dims.Omega[0], dims.Omega[1])
        self.table_bytes = dims.table_bytes
        self.device_bytes = dims.device_bytes
        order = np.empty(self.H, dtype=np.int32)
        _check(lib.egt_hand_order(self._h, order.ctypes.data))
        self.order = order

    def close(self):
        if getattr(self, "_h", None):
            _check(lib.egt_destroy_game(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- layout helpers (host-side marshalling between input hand order and [seq][ld]) ----
    def pack(self, arr):
        """[S][H] in input hand order -> [S][ld] numpy in sorted order (padding 0)."""
        arr = np.asarray(arr)
        out = np.zeros((arr.shape[0], self.ld), dtype=arr.dtype)
        out[:, :self.H] = arr[:, self.order]
        return out

    def unpack(self, arr):
        """[S][ld] in sorted order -> [S][H] in input hand order."""
        arr = np.asarray(arr)
        out = np.empty((arr.shape[0], self.H), dtype=arr.dtype)
        out[:, self.order] = arr[:, :self.H]
        return out

    def treeplex(self, player):
        J = self.J[player]
        par, first, n, lev = (np.empty(J, np.int32) for _ in range(4))
        beta = np.empty(J, np.float64)
        _check(lib.egt_treeplex_query(self._h, player, par.ctypes.data, first.ctypes.data,
                                      n.ctypes.data, lev.ctypes.data, beta.ctypes.data))
        return dict(parent=par, first=first, n=n, level=lev, beta=beta)

    def terminals(self):
        T = self.T
        s1, s2, kind = (np.empty(T, np.int32) for _ in range(3))
        coef = np.empty(T, np.float64)
        _check(lib.egt_terminal_query(self._h, s1.ctypes.data, s2.ctypes.data, kind.ctypes.data,
                                      coef.ctypes.data))
        return dict(seq1=s1, seq2=s2, kind=kind, coef=coef)

    # ---- hot path ----
    def grad(self, player, inp, out, stream=None):
        _check(lib.egt_grad(self._h, player, _ptr(inp), _ptr(out), _stream(stream)))

    def grad_f64(self, player, inp, out, stream=None):
        _check(lib.egt_grad_f64(self._h, player, _ptr(inp), _ptr(out), _stream(stream)))

    def smoothed_br(self, player, g, mu, q_out=None, value=True, stream=None):
        v = C.c_double(float("nan"))
        _check(lib.egt_smoothed_br(self._h, player, _ptr(g), float(mu), _ptr(q_out),
                                   C.byref(v) if value else None, _stream(stream)))
        return v.value if value else None

    def best_response_f64(self, player, g, stream=None):
        v = C.c_double()
        _check(lib.egt_best_response_f64(self._h, player, _ptr(g), C.byref(v), _stream(stream)))
        return v.value

    def gap(self, x, y, stream=None):
        v = C.c_double()
        _check(lib.egt_gap(self._h, _ptr(x), _ptr(y), C.byref(v), _stream(stream)))
        return v.value

    def gap_noalloc(self, x, y, stream=None):
        v = C.c_double()
        _check(lib.egt_gap_noalloc(self._h, _ptr(x), _ptr(y), C.byref(v), _stream(stream)))
        return v.value

    # ---- solver ----
    @staticmethod
    def _opts(variant=EGT_AS, alpha=0.01, mu0=None, eps_mbb=1.0, max_iters=1000, gap_every=1,
              replay=None, log_cap=0, engine=ENGINE_DEVICE):
        o = SolveOpts()
        o.variant, o.alpha = variant, alpha
        o.mu0[0], o.mu0[1] = (mu0 if mu0 is not None else (0.0, 0.0))
        o.eps_mbb, o.max_iters, o.gap_every = eps_mbb, max_iters, gap_every
        o.engine = engine
        keep = []
        if replay is not None and len(replay):
            pl = np.ascontiguousarray([p for p, _ in replay], dtype=np.int32)
            ta = np.ascontiguousarray([t for _, t in replay], dtype=np.float64)
            keep += [pl, ta]
            o.replay_n = len(replay)
            o.replay_player, o.replay_tau = _i32p(pl), _f64p(ta)
        log = None
        if log_cap:
            log = (IterLog * log_cap)()
            o.log_cap, o.log = log_cap, C.cast(log, C.POINTER(IterLog))
        return o, keep, log

    def solver_init(self, stream=None, **kw):
        o, keep, _ = self._opts(**kw)
        _check(lib.egt_solver_init(self._h, C.byref(o), _stream(stream)))

    def step(self, player=-1, tau=0.5, mode=STEP_DECR, stream=None):
        t = C.c_double(tau)
        info = StepInfo()
        _check(lib.egt_step(self._h, player, C.byref(t), mode, C.byref(info), _stream(stream)))
        return dict(player=info.player, accepted=bool(info.accepted), backoffs=info.backoffs,
                    products=info.products, tau=info.tau, egv=info.egv, mu=(info.mu[0], info.mu[1]))

    def step_point(self, v_hat, stream=None):
        """Copy the last egt_step attempt's intermediate point (x_hat or y_hat) into v_hat;
        returns the player it belongs to (egt_step_point)."""
        p = C.c_int32()
        _check(lib.egt_step_point(self._h, _ptr(v_hat), C.byref(p), _stream(stream)))
        return p.value

    def state_get(self, x=None, y=None, stream=None):
        mu = (C.c_double * 2)()
        _check(lib.egt_state_get(self._h, _ptr(x), _ptr(y), C.cast(mu, C.c_void_p), _stream(stream)))
        return (mu[0], mu[1])

    def state_set(self, x, y, mu, stream=None):
        m = (C.c_double * 2)(*mu)
        _check(lib.egt_state_set(self._h, _ptr(x), _ptr(y), C.cast(m, C.c_void_p), _stream(stream)))

    def checkpoint(self, x=None, y=None, stream=None):
        """Save the solve: iterates into x, y (device, may be None) and the scalars, returned as
        dict(t, tau, mu, gap_mbb) (egt_checkpoint_get)."""
        ck = Checkpoint()
        _check(lib.egt_checkpoint_get(self._h, _ptr(x), _ptr(y), C.byref(ck), _stream(stream)))
        return dict(t=ck.t, tau=ck.tau, mu=(ck.mu[0], ck.mu[1]), gap_mbb=ck.gap_mbb)

    def restore(self, x, y, scalars, stream=None):
        """Continue a saved solve (egt_checkpoint_set)."""
        ck = Checkpoint(scalars["t"], scalars["tau"], (C.c_double * 2)(*scalars["mu"]), scalars["gap_mbb"])
        _check(lib.egt_checkpoint_set(self._h, _ptr(x), _ptr(y), C.byref(ck), _stream(stream)))

    def save(self, path):
        """Checkpoint to a host .npz file: x, y ([S_p][ld] FP32) and the scalars."""
        import torch
        x = torch.empty((self.S[0], self.ld), device=f"cuda:{self.device}")
        y = torch.empty((self.S[1], self.ld), device=f"cuda:{self.device}")
        sc = self.checkpoint(x, y)
        torch.cuda.synchronize(self.device)
        np.savez(path, x=x.cpu().numpy(), y=y.cpu().numpy(), t=sc["t"], tau=sc["tau"],
                 mu=np.array(sc["mu"]), gap_mbb=sc["gap_mbb"])

    def load(self, path):
        """Continue the solve saved by save(path) on this game (same description)."""
        import torch
        d = np.load(path)
        if d["x"].shape != (self.S[0], self.ld) or d["y"].shape != (self.S[1], self.ld):
            raise EGTError(1, "checkpoint shapes do not match this game")
        x = torch.from_numpy(d["x"]).to(f"cuda:{self.device}")
        y = torch.from_numpy(d["y"]).to(f"cuda:{self.device}")
        self.restore(x, y, dict(t=int(d["t"]), tau=float(d["tau"]), mu=tuple(float(v) for v in d["mu"]),
                                gap_mbb=float(d["gap_mbb"])))
        torch.cuda.synchronize(self.device)

    ENGINE_PHASES = ("sbr_hat", "grad_1", "sbr_other", "grad_2", "sbr_tilde", "grad_3", "tail",
                     "decisions", "top")

    def engine_trace(self, reset=True):
        """Per-phase device time of the device-resident driver: total (us), CTA 0's
        own work (work_us), phases timed (n), average per phase (avg_us).  Recorded
        only while ``profile(1)`` is on for the game."""
        k = len(self.ENGINE_PHASES)
        us = np.zeros(k, np.float64)
        work = np.zeros(k, np.float64)
        n = np.zeros(k, np.int64)
        _check(lib.egt_engine_trace(self._h, int(reset), us.ctypes.data, work.ctypes.data, n.ctypes.data))
        return {name: dict(us=float(us[i]), work_us=float(work[i]), n=int(n[i]),
                           avg_us=float(us[i] / n[i]) if n[i] else 0.0,
                           avg_work_us=float(work[i] / n[i]) if n[i] else 0.0)
                for i, name in enumerate(self.ENGINE_PHASES)}

    def profile(self, enable):
        _check(lib.egt_profile(self._h, int(enable)))

    def profile_read(self):
        ms = np.zeros(len(KERNEL_KINDS), np.float64)
        n = np.zeros(len(KERNEL_KINDS), np.int64)
        _check(lib.egt_profile_read(self._h, ms.ctypes.data, n.ctypes.data))
        return {k: dict(ms=float(ms[i]), launches=int(n[i])) for i, k in enumerate(KERNEL_KINDS)}

    def iterate(self, n_iters, variant=EGT_AS, eps_mbb=0.0, gap_every=1, stream=None):
        o, keep, _ = self._opts(variant=variant, eps_mbb=eps_mbb, gap_every=gap_every)
        rep = SolveReport()
        _check(lib.egt_iterate(self._h, C.byref(o), int(n_iters), C.byref(rep), _stream(stream)))
        return dict(iters=rep.iters, products=rep.products, backoffs=rep.backoffs,
                    gap_checks=rep.gap_checks, gap_mbb=rep.gap_mbb, mu=(rep.mu[0], rep.mu[1]),
                    tau=rep.tau, seconds=rep.seconds)

    def state_gap(self, stream=None):
        v = C.c_double()
        _check(lib.egt_state_gap(self._h, C.byref(v), _stream(stream)))
        return v.value

    def solve(self, x_out=None, y_out=None, stream=None, raise_on_not_converged=False, **kw):
        o, keep, log = self._opts(**kw)
        rep = SolveReport()
        st = lib.egt_solve(self._h, C.byref(o), _ptr(x_out), _ptr(y_out), C.byref(rep), _stream(stream))
        if st != 0 and not (st == 6 and not raise_on_not_converged):
            _check(st)
        out = dict(status=STATUS[st], iters=rep.iters, products=rep.products, backoffs=rep.backoffs,
                   gap_checks=rep.gap_checks, gap_mbb=rep.gap_mbb, mu=(rep.mu[0], rep.mu[1]),
                   tau=rep.tau, seconds=rep.seconds)
        if log is not None:
            n = min(rep.iters, o.log_cap)
            out["log"] = [dict(t=log[i].t, player=log[i].player, backoffs=log[i].backoffs,
                               tau=log[i].tau, mu=(log[i].mu[0], log[i].mu[1]), egv=log[i].egv,
                               gap_mbb=log[i].gap_mbb, time_ns=log[i].time_ns) for i in range(n)]
        return out


class Batch:
    """Many games advanced together by one device-resident launch per step (egt_batch_*)."""

    def __init__(self, device=0):
        self._h = _vp()
        _check(lib.egt_batch_create(device, C.byref(self._h)))
        self.device = device
        self.members = {}

    def close(self):
        if getattr(self, "_h", None):
            _check(lib.egt_batch_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add(self, game, variant=EGT_AS, eps_mbb=1.0, max_iters=1000, gap_every=1):
        """Add an initialised game (Game.solver_init); returns its slot."""
        o, _, _ = Game._opts(variant=variant, eps_mbb=eps_mbb, max_iters=max_iters, gap_every=gap_every)
        slot = C.c_int32()
        _check(lib.egt_batch_add(self._h, game._h, C.byref(o), C.byref(slot)))
        self.members[slot.value] = game
        return slot.value

    def remove(self, slot):
        _check(lib.egt_batch_remove(self._h, slot))
        self.members.pop(slot, None)

    def step(self, n_iters, group=0, stream=None):
        """One launch; returns the number of members still active."""
        n = C.c_int32()
        _check(lib.egt_batch_step(self._h, n_iters, group, C.byref(n), _stream(stream)))
        return n.value

    def member(self, slot):
        m = BatchMemberInfo()
        _check(lib.egt_batch_member(self._h, slot, C.byref(m)))
        r = m.rep
        return dict(active=bool(m.active), status=STATUS[m.status], iters=r.iters, products=r.products,
                    backoffs=r.backoffs, gap_checks=r.gap_checks, gap_mbb=r.gap_mbb,
                    mu=(r.mu[0], r.mu[1]), tau=r.tau, seconds=r.seconds)

    def launch_shape(self):
        g, n = C.c_int32(), C.c_int32()
        _check(lib.egt_batch_launch_shape(self._h, C.byref(g), C.byref(n)))
        return g.value, n.value

    @property
    def shape(self):
        """The launch shape of group-0 steps: dict(share, pairs, grid_pct, pack, wave_mb, wave_min)."""
        x = LaunchShape()
        _check(lib.egt_batch_get_shape(self._h, C.byref(x)))
        return dict(share=x.share, pairs=x.pairs, grid_pct=x.grid_pct, pack=x.pack, wave_mb=x.wave_mb,
                    wave_min=x.wave_min)

    @shape.setter
    def shape(self, value):
        """Set some or all of the fields; the others keep their current values."""
        cur = self.shape
        cur.update(value)
        x = LaunchShape(cur["share"], cur["pairs"], cur["grid_pct"], cur["pack"], cur["wave_mb"], cur["wave_min"])
        _check(lib.egt_batch_set_shape(self._h, C.byref(x)))

    def tune(self, n_iters=20, reps=1, stream=None):
        """Autotune the launch shape on real steps of this batch (egt_batch_tune); returns the
        candidates with their time per member-iteration and the index of the one kept."""
        r = TuneReport()
        _check(lib.egt_batch_tune(self._h, n_iters, reps, C.byref(r), _stream(stream)))
        cands = [dict(share=r.shape[k].share, pairs=r.shape[k].pairs, grid_pct=r.shape[k].grid_pct,
                      pack=r.shape[k].pack, wave_mb=r.shape[k].wave_mb, wave_min=r.shape[k].wave_min,
                      us_per_iter=r.us_per_iter[k],
                      iters=r.iters[k]) for k in range(r.n)]
        return dict(best=r.best, candidates=cands)

    def run(self, n_iters=200, group=0, stream=None):
        """Step until no member is active; returns the number of steps taken."""
        steps = 0
        while True:
            steps += 1
            if self.step(n_iters, group, stream) == 0:
                return steps


class Server:
    """Continuous batching of solve requests on one device (egt_server_*)."""

    def __init__(self, device=0, mem_budget_bytes=0, max_running=0, iters_per_step=200, group=0):
        o = ServerOpts(mem_budget_bytes, max_running, iters_per_step, group)
        self._h = _vp()
        _check(lib.egt_server_create(device, C.byref(o), C.byref(self._h)))
        self.device = device

    def close(self):
        if getattr(self, "_h", None):
            _check(lib.egt_server_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def clock(self):
        return lib.egt_server_clock(self._h)

    def submit(self, spec, arrival=-1.0, variant=EGT_AS, alpha=0.01, eps_mbb=1.0, max_iters=20000,
               gap_every=1, mu0=None):
        d, keep = _desc(spec)
        o, _, _ = Game._opts(variant=variant, alpha=alpha, mu0=mu0, eps_mbb=eps_mbb, max_iters=max_iters,
                             gap_every=gap_every)
        rid = C.c_int64()
        _check(lib.egt_server_submit(self._h, C.byref(d), C.byref(o), float(arrival), C.byref(rid)))
        return rid.value

    def step(self, stream=None):
        st = ServerStats()
        _check(lib.egt_server_step(self._h, C.byref(st), _stream(stream)))
        return dict(queued=st.queued, running=st.running, completed=st.completed, launches=st.launches,
                    used_bytes=st.used_bytes, budget_bytes=st.budget_bytes, clock=st.clock)

    def result(self, rid, release=True, iterates=True):
        """State of a request; once done also its iterates (host numpy [S][ld]) and report."""
        info = ServerRequestInfo()
        _check(lib.egt_server_result(self._h, rid, C.byref(info), None, None, 0))
        out = dict(state=lib.egt_server_state_name(info.state).decode(), status=STATUS[info.status],
                   t_submit=info.t_submit, t_admit=info.t_admit, t_done=info.t_done)
        if info.state == 2:
            r = info.rep
            out.update(iters=r.iters, products=r.products, backoffs=r.backoffs, gap_mbb=r.gap_mbb,
                       mu=(r.mu[0], r.mu[1]), tau=r.tau, latency=info.t_done - info.t_submit)
            x = y = None
            if iterates:
                x = np.empty((info.S[0], info.ld), np.float32)
                y = np.empty((info.S[1], info.ld), np.float32)
            _check(lib.egt_server_result(self._h, rid, C.byref(info),
                                         x.ctypes.data if x is not None else None,
                                         y.ctypes.data if y is not None else None, int(release)))
            out.update(x=x, y=y)
        return out
