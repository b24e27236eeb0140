"""GB300 implementation of the GENGA long-range kick path (Brasser et al. 2023).

A thin ctypes binding over ``libgenga.so`` (C ABI in ``include/genga.h``).
The functions below carry the C names and only marshal arguments; every step
of the path runs in the library's CUDA kernels.  PyTorch provides the device
memory and streams.  Loading fails loudly when the library is missing: there
is no CPU fallback.

    import paper_2309_08217_gb300 as g
    g.build()                                  # nvcc, sm_103a, in-tree
    ctx = g.genga_create(max_N=40_000)
    sys = g.DeviceSystem.from_disc(disc)       # float64 tensors on cuda
    p = g.make_params(G=disc.G, Mstar=1.0, dt=6.0, precision=g.GENGA_FP32)
    g.genga_kick(ctx, sys, p, tau=3.0, acc=acc_tensor)
    # hybrid steps with the close-encounter level and tuned intermediate levels
    p = g.make_params(G=disc.G, Mstar=1.0, dt=6.0, precision=g.GENGA_FP32, bs_tol=1e-12)
    (p.n_levels, p.n_sub), ms = g.genga_tune_levels(ctx, sys, p, [(0, 2), (2, 3), (2, 4)])
    g.genga_step(ctx, sys, p, 1000)
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import discs  # noqa: F401  (seeded inputs; numpy only)

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgenga.so")

GENGA_OK, GENGA_ERR_INVALID_ARG, GENGA_ERR_CUDA, GENGA_ERR_CAPACITY = 0, 1, 2, 3
GENGA_ERR_KEPLER, GENGA_ERR_NONFINITE, GENGA_ERR_TIMEOUT, GENGA_ERR_BS = 4, 5, 6, 7
GENGA_FP64, GENGA_FP32_HILO, GENGA_FP32_BLOCKREL, GENGA_FP32 = 0, 1, 2, 3
GENGA_RCRIT_EQ1, GENGA_RCRIT_MUTUAL_HILL = 0, 1
GENGA_K_CHAMBERS, GENGA_K_QUINTIC = 0, 1


class genga_params(C.Structure):
    _fields_ = [("G", C.c_double), ("Mstar", C.c_double), ("dt", C.c_double),
                ("n1", C.c_double), ("n2", C.c_double),
                ("rcrit_mode", C.c_int32), ("changeover", C.c_int32),
                ("precision", C.c_int32), ("kepler_max_iter", C.c_int32), ("n_big", C.c_int32),
                ("bs_tol", C.c_double), ("r_in", C.c_double), ("r_out", C.c_double),
                ("n_levels", C.c_int32), ("n_sub", C.c_int32)]


class genga_system(C.Structure):
    _fields_ = [("N", C.c_int32)] + [(n, C.c_void_p) for n in ("x", "y", "z", "vx", "vy", "vz", "m", "radius")]


class GengaError(RuntimeError):
    def __init__(self, code, where=""):
        self.code = int(code)
        extra = ""
        if self.code == GENGA_ERR_CUDA and _lib is not None:
            extra = f", {_lib.genga_last_cuda_error().decode()}"
        super().__init__(f"{where}: {genga_status_string(code)} (code {code}{extra})")


_lib = None
_lock = threading.Lock()


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libgenga.so for sm_103a (nvcc) into the package directory."""
    from .nvcc_build import build as _b  # (a submodule named "build" would replace this function on import)
    return _b(force=force, verbose=verbose)


def load():
    """Load libgenga.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libgenga.so not found at {LIB_PATH}: run paper_2309_08217_gb300.build()")
        lib = C.CDLL(LIB_PATH)
        P, S, V, I, D = C.POINTER(genga_params), C.POINTER(genga_system), C.c_void_p, C.c_int32, C.c_double
        sigs = {
            "genga_create": ([C.POINTER(V), I, I], I),
            "genga_destroy": ([V], None),
            "genga_kick": ([V, S, P, D, V, V], I),
            "genga_drift": ([V, S, P, D, V], I),
            "genga_encounters": ([V, S, P, V, I, V, V], I),
            "genga_last_encounters": ([V, V, I, V, V], I),
            "genga_step": ([V, S, P, I, V], I),
            "genga_energy": ([V, S, P, C.POINTER(C.c_double), V], I),
            "genga_get_status": ([V, V], I),
            "genga_status_string": ([I], C.c_char_p),
            "genga_profile_enable": ([V, I], I),
            "genga_profile_read": ([V, C.POINTER(C.c_double), C.POINTER(C.c_int32), I], I),
            "genga_measure_alu_peaks": ([I, C.POINTER(C.c_double), C.POINTER(C.c_double)], I),
            "genga_set_kernel_variant": ([V, I], I),
            "genga_set_test_waits": ([V, I, I], I),
            "genga_last_cuda_error": ([], C.c_char_p),
            "genga_kernel_variant_info": ([I] + [C.POINTER(I)] * 4, I),
            "genga_set_step_graphs": ([V, I], I),
            "genga_kick_noalloc": ([S, P, D, V, V], I),
            "genga_measure_fma2_peak": ([I, C.POINTER(C.c_double)], I),
            "genga_launch_count": ([V, C.POINTER(C.c_int64)], I),
            "genga_kick_batched": ([V, S, C.POINTER(C.c_int32), I, P, D, V, V], I),
            "genga_tuning_times": ([V, I, C.POINTER(C.c_float), I], I),
            "genga_step_batched": ([V, S, C.POINTER(C.c_int32), I, P, I, V], I),
            "genga_get_kernel_variant": ([V, I, C.POINTER(C.c_int32), C.POINTER(C.c_int32)], I),
            "genga_set_fp64_variant": ([V, I], I),
            "genga_mutual_plan_check": ([I, C.POINTER(C.c_int32), I, I, I, C.POINTER(C.c_int64)], I),
            "genga_batched_tuning": ([V, C.POINTER(C.c_int32), I, C.POINTER(C.c_int32), C.POINTER(C.c_float), I], I),
            "genga_get_fp64_variant": ([V, I, C.POINTER(C.c_int32), C.POINTER(C.c_int32)], I),
            "genga_fp64_variant_info": ([I] + [C.POINTER(I)] * 3, I),
            "genga_fp64_tuning_times": ([V, I, C.POINTER(C.c_float), I], I),
            "genga_compact": ([V, S, V, V], I),
            "genga_tune_levels": ([V, S, P, C.POINTER(I), C.POINTER(I), I, I, C.POINTER(I), C.POINTER(C.c_float),
                                   C.POINTER(I), V], I),
        }
        for name, (args, res) in sigs.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
        return lib


def genga_status_string(code) -> str:
    return load().genga_status_string(int(code)).decode()


def _check(code, where):
    if code != GENGA_OK:
        raise GengaError(code, where)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def make_params(G, Mstar=1.0, dt=6.0, n1=3.0, n2=0.4, rcrit_mode=GENGA_RCRIT_MUTUAL_HILL,
                changeover=GENGA_K_CHAMBERS, precision=GENGA_FP32, kepler_max_iter=50, n_big=-1,
                bs_tol=0.0, r_in=0.0, r_out=0.0, n_levels=0, n_sub=2) -> genga_params:
    """n_big >= 0: test-particle mode 2 (bodies n_big.. feel the first n_big bodies, not each other).
    bs_tol > 0: the drift integrates the close-encounter groups (Bulirsch-Stoer, that tolerance).
    r_in, r_out > 0: removal radii (bodies inside / beyond become ghosts after each drift).
    n_levels > 0 (with bs_tol > 0): that many intermediate levels of n_sub sub-steps."""
    return genga_params(G, Mstar, dt, n1, n2, rcrit_mode, changeover, precision, kepler_max_iter, n_big,
                        bs_tol, r_in, r_out, n_levels, n_sub)


class DeviceSystem:
    """Seven float64 CUDA tensors (x, y, z, vx, vy, vz, m), optional physical
    radii, and their genga_system view."""

    def __init__(self, x, y, z, vx, vy, vz, m, radius=None):
        self.tensors = [x, y, z, vx, vy, vz, m]
        self.radius = radius
        for t in self.tensors + ([radius] if radius is not None else []):
            if not (t.is_cuda and t.dtype.is_floating_point and t.element_size() == 8 and t.is_contiguous()):
                raise ValueError("state arrays must be contiguous float64 CUDA tensors")
        self.c = genga_system(int(m.numel()), *[t.data_ptr() for t in self.tensors],
                              radius.data_ptr() if radius is not None else None)

    @property
    def N(self):
        return int(self.c.N)

    @classmethod
    def from_disc(cls, disc, device="cuda", radius=None):
        import torch
        r = None if radius is None else torch.tensor(radius, dtype=torch.float64, device=device)
        return cls(*[torch.tensor(a, dtype=torch.float64, device=device) for a in disc.arrays()], radius=r)

    @classmethod
    def from_arrays(cls, arrays, device="cuda", radius=None):
        import torch
        r = None if radius is None else torch.as_tensor(radius, dtype=torch.float64).to(device).contiguous()
        return cls(*[torch.as_tensor(a, dtype=torch.float64).to(device).contiguous() for a in arrays], radius=r)

    def numpy(self):
        """The N current bodies' seven arrays (after genga_compact: the first N entries)."""
        n = self.N
        return [t.detach()[:n].cpu().numpy().copy() for t in self.tensors]

    def radius_numpy(self):
        return None if self.radius is None else self.radius.detach()[: self.N].cpu().numpy().copy()


class Context:
    """Owns a genga_ctx (workspace for up to max_N bodies on one device)."""

    def __init__(self, max_N, device=0):
        self.ptr = genga_create(max_N, device)

    def close(self):
        if self.ptr:
            genga_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------- C-ABI names ---
def genga_create(max_N, device=0):
    h = C.c_void_p()
    _check(load().genga_create(C.byref(h), int(max_N), int(device)), "genga_create")
    return h


def genga_destroy(ctx):
    load().genga_destroy(ctx.ptr if isinstance(ctx, Context) else ctx)


def _ctx(ctx):
    return ctx.ptr if isinstance(ctx, Context) else ctx


def _sys(sys):
    return C.byref(sys.c if isinstance(sys, DeviceSystem) else sys)


def genga_kick(ctx, sys, params, tau=0.0, acc=None, stream=None):
    _check(load().genga_kick(_ctx(ctx), _sys(sys), C.byref(params), float(tau), _ptr(acc), _stream(stream)),
           "genga_kick")


def genga_drift(ctx, sys, params, dt, stream=None):
    _check(load().genga_drift(_ctx(ctx), _sys(sys), C.byref(params), float(dt), _stream(stream)), "genga_drift")


def genga_encounters(ctx, sys, params, pairs, capacity, count, stream=None):
    _check(load().genga_encounters(_ctx(ctx), _sys(sys), C.byref(params), _ptr(pairs), int(capacity),
                                   _ptr(count), _stream(stream)), "genga_encounters")


def genga_last_encounters(ctx, pairs, capacity, count, stream=None):
    _check(load().genga_last_encounters(_ctx(ctx), _ptr(pairs), int(capacity), _ptr(count), _stream(stream)),
           "genga_last_encounters")


def genga_step(ctx, sys, params, nsteps, stream=None):
    _check(load().genga_step(_ctx(ctx), _sys(sys), C.byref(params), int(nsteps), _stream(stream)), "genga_step")


def _offsets(offsets):
    arr = (C.c_int32 * len(offsets))(*[int(v) for v in offsets])
    return arr, len(offsets) - 1


def genga_kick_batched(ctx, all_sys, offsets, params, tau=0.0, acc=None, stream=None):
    """Kick of D independent systems concatenated in all_sys (offsets: D+1 ints)."""
    off, D = _offsets(offsets)
    _check(load().genga_kick_batched(_ctx(ctx), _sys(all_sys), off, D, C.byref(params), float(tau), _ptr(acc),
                                     _stream(stream)), "genga_kick_batched")


def genga_step_batched(ctx, all_sys, offsets, params, nsteps, stream=None):
    """nsteps level-0 steps of D independent systems concatenated in all_sys."""
    off, D = _offsets(offsets)
    _check(load().genga_step_batched(_ctx(ctx), _sys(all_sys), off, D, C.byref(params), int(nsteps),
                                     _stream(stream)), "genga_step_batched")


def genga_energy(ctx, sys, params, stream=None):
    out = (C.c_double * 4)()
    _check(load().genga_energy(_ctx(ctx), _sys(sys), C.byref(params), out, _stream(stream)), "genga_energy")
    return list(out)


def genga_compact(ctx, sys, id=None, stream=None) -> int:
    """Remove the ghosts (merged or removed bodies) from sys's arrays, keeping the
    others in order (and id, an optional int32 CUDA tensor, along); returns the
    new N (sys's view is updated)."""
    _check(load().genga_compact(_ctx(ctx), _sys(sys), _ptr(id), _stream(stream)), "genga_compact")
    return int((sys.c if isinstance(sys, DeviceSystem) else sys).N)


def genga_tune_levels(ctx, sys, params, candidates, trial_steps=8, stream=None, codes=None):
    """Time trial steps of each (n_levels, n_sub) in `candidates` from a copy of
    sys's state (left unchanged); returns (the fastest pair whose trial raised
    no status, ms per step of each).  codes: optional list, extended with each
    candidate's status code."""
    cand = list(candidates)
    nl = (C.c_int32 * len(cand))(*[int(c[0]) for c in cand])
    ns = (C.c_int32 * len(cand))(*[int(c[1]) for c in cand])
    best = C.c_int32(-1)
    ms = (C.c_float * len(cand))()
    cs = (C.c_int32 * len(cand))()
    _check(load().genga_tune_levels(_ctx(ctx), _sys(sys), C.byref(params), nl, ns, len(cand), int(trial_steps),
                                    C.byref(best), ms, cs, _stream(stream)), "genga_tune_levels")
    if codes is not None:
        codes.extend(int(v) for v in cs)
    return tuple(cand[best.value]), [float(v) for v in ms]


def genga_get_status(ctx, stream=None) -> int:
    """Synchronise, return and clear the sticky device status (an int code)."""
    return int(load().genga_get_status(_ctx(ctx), _stream(stream)))


# ------------------------------------------------- measurement hooks ------
def genga_profile_enable(ctx, enable=True):
    _check(load().genga_profile_enable(_ctx(ctx), 1 if enable else 0), "genga_profile_enable")


def genga_profile_read(ctx, reset=True):
    """(summed device ms, number) of the long-range pass launches recorded."""
    ms, n = C.c_double(), C.c_int32()
    _check(load().genga_profile_read(_ctx(ctx), C.byref(ms), C.byref(n), 1 if reset else 0),
           "genga_profile_read")
    return ms.value, n.value


def genga_measure_alu_peaks(device=0):
    """Measured FFMA and DFMA throughput of `device` in TFLOP/s."""
    f32, f64 = C.c_double(), C.c_double()
    _check(load().genga_measure_alu_peaks(int(device), C.byref(f32), C.byref(f64)), "genga_measure_alu_peaks")
    return f32.value, f64.value


def genga_launch_count(ctx):
    """Kernels the context has launched so far."""
    n = C.c_int64()
    _check(load().genga_launch_count(_ctx(ctx), C.byref(n)), "genga_launch_count")
    return n.value


def genga_measure_fma2_peak(device=0):
    """Measured packed two-lane FP32 FMA throughput of `device` in TFLOP/s."""
    t = C.c_double()
    _check(load().genga_measure_fma2_peak(int(device), C.byref(t)), "genga_measure_fma2_peak")
    return t.value


def genga_tuning_times(ctx, N):
    """The autotuner's pass time (ms) of each FP32 variant for N bodies."""
    n = genga_get_kernel_variant(ctx, N)[1]
    arr = (C.c_float * n)()
    _check(load().genga_tuning_times(_ctx(ctx), int(N), arr, n), "genga_tuning_times")
    return list(arr)


def genga_set_step_graphs(ctx, enable=True):
    """Replay captured 4-step graphs in genga_step / genga_step_batched (default) or not."""
    _check(load().genga_set_step_graphs(_ctx(ctx), int(bool(enable))), "genga_set_step_graphs")


def genga_set_kernel_variant(ctx, variant=-1):
    """Force an FP32 pass variant (>= 0) or return to autotuning (-1)."""
    _check(load().genga_set_kernel_variant(_ctx(ctx), int(variant)), "genga_set_kernel_variant")


def genga_kernel_variant_info(variant):
    """{'kind': 0 one-sided / 1 mutual, 'warps', 'bodies_per_thread', 'ctas_per_sm'} of an FP32 variant."""
    vals = [C.c_int32() for _ in range(4)]
    _check(load().genga_kernel_variant_info(int(variant), *[C.byref(v) for v in vals]), "genga_kernel_variant_info")
    return dict(zip(("kind", "warps", "bodies_per_thread", "ctas_per_sm"), (v.value for v in vals)))


def genga_set_test_waits(ctx, wait_ns_log2=0, hold=False):
    """Test hook of the pipelined passes' bounded waits: limit 2^wait_ns_log2 ns
    (0: the default 2 s); hold: the producers withhold their first stage."""
    _check(load().genga_set_test_waits(_ctx(ctx), int(wait_ns_log2), int(bool(hold))), "genga_set_test_waits")


def genga_get_kernel_variant(ctx, N):
    """(variant in use for N bodies or -1 if not tuned yet, number of variants)."""
    v, n = C.c_int32(), C.c_int32()
    _check(load().genga_get_kernel_variant(_ctx(ctx), int(N), C.byref(v), C.byref(n)), "genga_get_kernel_variant")
    return v.value, n.value


def genga_batched_tuning(ctx, offsets):
    """(FP32 variant tuned for this batch layout or -1, batched pass ms of each one-sided variant)."""
    off, D = _offsets(offsets)
    n = genga_get_kernel_variant(ctx, 1)[1]
    v, arr = C.c_int32(), (C.c_float * n)()
    _check(load().genga_batched_tuning(_ctx(ctx), off, D, C.byref(v), arr, n), "genga_batched_tuning")
    return v.value, list(arr)


def genga_mutual_plan_check(sizes, cw, npg, ctas=152):
    """Host-only check of the mutual work plan for systems of the given sizes;
    returns (items, largest rows of a system, group-pair visits, row entries)."""
    n = (C.c_int32 * len(sizes))(*[int(v) for v in sizes])
    st = (C.c_int64 * 4)()
    _check(load().genga_mutual_plan_check(len(sizes), n, int(cw), int(npg), int(ctas), st), "genga_mutual_plan_check")
    return tuple(st)


def genga_set_fp64_variant(ctx, variant=-1):
    """Force an FP64 pass variant (0 one-sided, >= 1 mutual) or return to autotuning (-1)."""
    _check(load().genga_set_fp64_variant(_ctx(ctx), int(variant)), "genga_set_fp64_variant")


def genga_get_fp64_variant(ctx, N):
    """(FP64 variant in use for N bodies or -1 if not tuned yet, number of FP64 variants)."""
    v, n = C.c_int32(), C.c_int32()
    _check(load().genga_get_fp64_variant(_ctx(ctx), int(N), C.byref(v), C.byref(n)), "genga_get_fp64_variant")
    return v.value, n.value


def genga_fp64_variant_info(variant):
    """{'kind': 0 one-sided / 1 mutual, 'warps', 'bodies_per_thread'} of an FP64 variant."""
    vals = [C.c_int32() for _ in range(3)]
    _check(load().genga_fp64_variant_info(int(variant), *[C.byref(v) for v in vals]), "genga_fp64_variant_info")
    return dict(zip(("kind", "warps", "bodies_per_thread"), (v.value for v in vals)))


def genga_fp64_tuning_times(ctx, N):
    """The autotuner's pass time (ms) of each FP64 variant for N bodies."""
    n = genga_get_fp64_variant(ctx, N)[1]
    arr = (C.c_float * n)()
    _check(load().genga_fp64_tuning_times(_ctx(ctx), int(N), arr, n), "genga_fp64_tuning_times")
    return list(arr)


# ------------------------------------------- kick without device allocation ---
GENGA_NOALLOC_MAX_N = 65536


def genga_kick_noalloc(sys, params, tau=0.0, acc=None, stream=None):
    """FP64 kick on the current device with no device allocation (its scratch
    is a fixed array inside the library; at most GENGA_NOALLOC_MAX_N bodies;
    overlapping calls race on that scratch)."""
    _check(load().genga_kick_noalloc(_sys(sys), C.byref(params), float(tau), _ptr(acc), _stream(stream)),
           "genga_kick_noalloc")
