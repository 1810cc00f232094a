"""Thin Python binding of the C ABI in include/sc.h (libsc.so).

Argument marshalling only: every step of the sweep runs in the library's CUDA
kernels.  The functions keep the C names; ``Context`` bundles them for one
grain.  Device buffers are torch tensors (plumbing: memory and streams).
If the compiled library is missing this module raises on import -- there is
no fallback path.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# SC_LIBRARY=checked selects the bounds-checked build (libsc_checked.so)
LIB_PATH = os.path.join(_HERE, "_lib", "libsc_checked.so" if os.environ.get("SC_LIBRARY") == "checked"
                        else "libsc.so")

SC_OK, SC_EINVAL, SC_ENOMEM, SC_ECUDA, SC_ETIMEOUT, SC_ENUMERIC, SC_ESTATE, SC_ENOTCONV = range(8)
STATUS_NAMES = ["SC_OK", "SC_EINVAL", "SC_ENOMEM", "SC_ECUDA", "SC_ETIMEOUT", "SC_ENUMERIC",
                "SC_ESTATE", "SC_ENOTCONV"]
SC_PREC_FP64, SC_PREC_FP32 = 0, 1
# sc_stepper: integrator of the Riccati equation along a line (App. C)
SC_STEP_CLOSED, SC_STEP_MIDPOINT = 0, 1
STEPPERS = {"closed": SC_STEP_CLOSED, "midpoint": SC_STEP_MIDPOINT}
# sc_energy_sum: energies and weights of the Matsubara sums (Sec. 3.1)
SC_SUM_MATSUBARA, SC_SUM_OZAKI = 0, 1
ENERGY_SUMS = {"matsubara": SC_SUM_MATSUBARA, "ozaki": SC_SUM_OZAKI}


class ScError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


class sc_part(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32), ("add", ctypes.c_int32),
        ("cx", ctypes.c_double), ("cy", ctypes.c_double), ("r", ctypes.c_double),
        ("n_vert", ctypes.c_int32),
        ("vx", ctypes.POINTER(ctypes.c_double)), ("vy", ctypes.POINTER(ctypes.c_double)),
    ]


class sc_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("h", ctypes.c_double), ("x0", ctypes.c_double), ("y0", ctypes.c_double),
        ("shape_kind", ctypes.c_int32),
        ("disc_cx", ctypes.c_double), ("disc_cy", ctypes.c_double), ("disc_r", ctypes.c_double),
        ("n_vert", ctypes.c_int32),
        ("vx", ctypes.POINTER(ctypes.c_double)), ("vy", ctypes.POINTER(ctypes.c_double)),
        ("pairing", ctypes.c_int32), ("crystal_rotation", ctypes.c_double),
        ("t", ctypes.c_double), ("flux_quanta", ctypes.c_double),
        ("gauge_cx", ctypes.c_double), ("gauge_cy", ctypes.c_double),
        ("kappa", ctypes.c_double), ("charge_sign", ctypes.c_int32),
        ("n_angles", ctypes.c_int32), ("n_energies", ctypes.c_int32),
        ("lattice_ox", ctypes.c_double), ("lattice_oy", ctypes.c_double),
        ("precision", ctypes.c_int32), ("lanes_per_line", ctypes.c_int32),
        ("host_only", ctypes.c_int32), ("record_timings", ctypes.c_int32),
        ("stepper", ctypes.c_int32), ("energy_sum", ctypes.c_int32),
        ("n_components", ctypes.c_int32), ("pairings", ctypes.c_int32 * 4), ("tc_ratios", ctypes.c_double * 4),
        ("n_parts", ctypes.c_int32), ("parts", ctypes.POINTER(sc_part)),
        ("gauge", ctypes.c_int32),
        ("eps_cut", ctypes.c_double), ("mask", ctypes.POINTER(ctypes.c_uint8)),
        ("adjoint_checkpoint", ctypes.c_int32),
    ]


GAUGES = {"symmetric": 0, "landau": 1, "solenoid": 2}
PART_KINDS = {"disc": 0, "polygon": 1}


class sc_batch_info(ctypes.Structure):
    _fields_ = [
        ("n_grains", ctypes.c_int32), ("n_items", ctypes.c_int32),
        ("energies_per_lane", ctypes.c_int32), ("steps_per_sweep", ctypes.c_int64),
        ("scratch_bytes", ctypes.c_int64), ("ms_sweep", ctypes.c_double),
        ("lane_steps_per_sweep", ctypes.c_int64), ("sweep_launches", ctypes.c_int32),
        ("class_ept", ctypes.c_int32 * 16), ("class_blocks_per_sm", ctypes.c_int32 * 16),
        ("class_ms", ctypes.c_double * 16), ("min_lanes_per_line", ctypes.c_int32),
        ("launches_per_iteration", ctypes.c_int32), ("split_members", ctypes.c_int32),
        ("split_ms_on", ctypes.c_double), ("split_ms_off", ctypes.c_double),
        ("fused_transfers", ctypes.c_int32), ("transfer_items", ctypes.c_int64),
        ("fuse_ms_on", ctypes.c_double), ("fuse_ms_off", ctypes.c_double),
        ("ms_iteration", ctypes.c_double),
    ]


class sc_info(ctypes.Structure):
    _fields_ = [
        ("n_pairs", ctypes.c_int32), ("n_lines", ctypes.c_int32),
        ("n_samples", ctypes.c_int64), ("n_in", ctypes.c_int64),
        ("steps_per_sweep", ctypes.c_int64), ("points_per_sweep", ctypes.c_int64),
        ("area", ctypes.c_double), ("norm_D", ctypes.c_double),
        ("lanes_per_line", ctypes.c_int32), ("energies_per_lane", ctypes.c_int32),
        ("lines_per_warp", ctypes.c_int32), ("scratch_bytes", ctypes.c_int64),
        ("ms_rotate", ctypes.c_double), ("ms_sweep", ctypes.c_double),
        ("ms_rotate_back", ctypes.c_double), ("ms_adjoint", ctypes.c_double),
    ]


class sc_accel_params(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32), ("step_size", ctypes.c_double), ("drag", ctypes.c_double),
        ("step_size_factor", ctypes.c_double), ("cos_similarity_min", ctypes.c_double),
        ("step_size_max", ctypes.c_double), ("step_size_min", ctypes.c_double),
    ]


# sc_accel_kind (App. E)
SC_ACC_PICARD, SC_ACC_POLYAK, SC_ACC_BARZILAI_BORWEIN, SC_ACC_CONGACC = 0, 1, 2, 3
ACCELERATORS = {"picard": SC_ACC_PICARD, "polyak": SC_ACC_POLYAK,
                "barzilai-borwein": SC_ACC_BARZILAI_BORWEIN, "congacc": SC_ACC_CONGACC}

# every symbol include/sc.h declares
EXPORTED = ["sc_params_default", "sc_create", "sc_destroy", "sc_get_info", "sc_get_mask",
            "sc_set_fields", "sc_get_fields", "sc_reset_boundary", "sc_riccati_sweep", "sc_burnin",
            "sc_gap_update", "sc_current", "sc_free_energy", "sc_update_vector_potential",
            "sc_picard_step", "sc_ldos", "sc_debug_lines", "sc_debug_ghost", "sc_debug_links", "sc_debug_chords",
            "sc_debug_exits", "sc_debug_images", "sc_debug_fp64_math", "sc_debug_fma_rate", "sc_debug_validate_tables",
            "sc_debug_corrupt_table", "sc_debug_bounds", "sc_sweep_lines_noalloc", "sc_sweep_adjoint",
            "sc_ldos_adjoint", "sc_accel_params_default", "sc_accelerate", "sc_accel_reset",
            "sc_accel_get_state", "sc_self_consistency", "sc_get_history", "sc_clear_history", "sc_ozaki_poles", "sc_ozaki_poles_for_cutoff", "sc_energy_grid",
            "sc_batch_create",
            "sc_batch_destroy", "sc_batch_member", "sc_batch_sweep", "sc_batch_run", "sc_batch_reset_boundary",
            "sc_batch_set_energy_parts", "sc_batch_set_fused_transfers",
            "sc_batch_autotune",
            "sc_batch_get_info", "sc_batch_set_fields", "sc_batch_get_outputs", "sc_last_error", "sc_version"]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libsc.so not built ({LIB_PATH}); run python -m paper_2205_15000_b300.build")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    P = ctypes.POINTER
    sig = {
        "sc_params_default": [P(sc_params)],
        "sc_create": [P(sc_params), P(vp)],
        "sc_destroy": [vp],
        "sc_get_info": [vp, P(sc_info)],
        "sc_get_mask": [vp, vp],
        "sc_set_fields": [vp, vp, vp, ctypes.c_int, vp],
        "sc_get_fields": [vp, vp, vp, ctypes.c_int, vp],
        "sc_reset_boundary": [vp],
        "sc_riccati_sweep": [vp, vp],
        "sc_burnin": [vp, i32, f64, vp],
        "sc_gap_update": [vp, vp, P(f64), ctypes.c_int, vp],
        "sc_current": [vp, vp, ctypes.c_int, vp],
        "sc_free_energy": [vp, P(f64), vp, ctypes.c_int, vp],
        "sc_update_vector_potential": [vp, vp],
        "sc_picard_step": [vp, vp],
        "sc_ldos": [vp, vp, i32, f64, i32, vp, ctypes.c_int, vp],
        "sc_debug_lines": [vp, vp, vp, vp, vp, vp, vp],
        "sc_debug_ghost": [vp, vp],
        "sc_debug_links": [vp, vp, vp, vp, vp],
        "sc_debug_chords": [vp, vp, vp],
        "sc_debug_exits": [vp, vp],
        "sc_debug_images": [vp, vp],
        "sc_debug_fp64_math": [vp, i64, vp, vp, vp],
        "sc_debug_fma_rate": [i32, P(f64), vp],
        "sc_debug_validate_tables": [vp, P(i64)],
        "sc_debug_corrupt_table": [vp, i32],
        "sc_debug_bounds": [P(ctypes.c_uint64), P(i32), i32],
        "sc_sweep_lines_noalloc": [vp, vp, vp, vp, vp, i32, i32, i32, f64, f64, vp, vp, vp],
        "sc_sweep_adjoint": [vp, vp, vp, vp, f64, vp, vp, ctypes.c_int, vp],
        "sc_ldos_adjoint": [vp, vp, i32, f64, i32, vp, vp, vp, ctypes.c_int, vp],
        "sc_ozaki_poles": [i32, vp, vp],
        "sc_self_consistency": [vp, P(sc_accel_params), i32, f64, i32, P(i32), P(f64), vp],
        "sc_get_history": [vp, P(i32), vp, vp],
        "sc_clear_history": [vp],
        "sc_ozaki_poles_for_cutoff": [f64, f64],
        "sc_energy_grid": [vp, vp, vp],
        "sc_accel_params_default": [i32, P(sc_accel_params)],
        "sc_accelerate": [vp, P(sc_accel_params), vp],
        "sc_accel_reset": [vp],
        "sc_accel_get_state": [vp, P(i32), vp, vp],
        "sc_batch_create": [vp, i32, i32, P(vp)],
        "sc_batch_destroy": [vp],
        "sc_batch_member": [vp, i32, P(vp)],
        "sc_batch_sweep": [vp, vp],
        "sc_batch_run": [vp, i32, i32, vp],
        "sc_batch_reset_boundary": [vp],
        "sc_batch_set_energy_parts": [vp, i32],
        "sc_batch_set_fused_transfers": [vp, i32],
        "sc_batch_autotune": [vp, P(i32), vp],
        "sc_batch_get_info": [vp, P(sc_batch_info)],
        "sc_batch_set_fields": [vp, vp, ctypes.c_int, vp],
        "sc_batch_get_outputs": [vp, vp, vp, vp, ctypes.c_int, vp],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    L.sc_last_error.argtypes = [vp]
    L.sc_last_error.restype = ctypes.c_char_p
    L.sc_version.argtypes = []
    L.sc_version.restype = ctypes.c_char_p
    return L


lib = _load()


def _check(st, ctx=None):
    if st != SC_OK:
        raise ScError(st, lib.sc_last_error(ctx).decode())


def _ptr(a):
    """Address of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(ctypes.c_void_p)
    return ctypes.c_void_p(a.data_ptr())


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except Exception:
            pass
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def sc_version():
    return lib.sc_version().decode()


def sc_params_default():
    p = sc_params()
    _check(lib.sc_params_default(ctypes.byref(p)))
    return p


def make_params(d, precision="fp32", lanes_per_line=0, host_only=False, record_timings=False):
    """sc_params from a workload dict (keys of workloads.PARAM_KEYS).  The
    vertex arrays are kept alive on the returned struct."""
    p = sc_params_default()
    for k in ("nx", "ny", "h", "x0", "y0", "shape_kind", "disc_cx", "disc_cy", "disc_r", "pairing",
              "crystal_rotation", "t", "flux_quanta", "gauge_cx", "gauge_cy", "kappa", "charge_sign",
              "n_angles", "n_energies", "lattice_ox", "lattice_oy"):
        setattr(p, k, d[k])
    vx = np.ascontiguousarray(d.get("vx", []) or [0.0], np.float64)
    vy = np.ascontiguousarray(d.get("vy", []) or [0.0], np.float64)
    p.n_vert = len(d.get("vx", [])) if d["shape_kind"] == 1 else 0
    p.vx = vx.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    p.vy = vy.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    p._keep = (vx, vy)
    p.precision = SC_PREC_FP64 if precision == "fp64" else SC_PREC_FP32
    p.lanes_per_line = lanes_per_line
    p.host_only = 1 if host_only else 0
    p.record_timings = 1 if record_timings else 0
    p.stepper = STEPPERS[d.get("stepper", "closed")]
    p.energy_sum = ENERGY_SUMS[d.get("energy_sum", "matsubara")]
    comps = d.get("components")
    if comps:  # [(pairing, T_c^Gamma / T_c), ...]; component 0 takes the place of `pairing`
        p.n_components = len(comps)
        p.pairing = int(comps[0][0])
        for c, (pairing, tcr) in enumerate(comps):
            p.pairings[c] = int(pairing)
            p.tc_ratios[c] = float(tcr)
    p.gauge = GAUGES[d.get("gauge", "symmetric")]
    parts = d.get("parts") or []
    arr = (sc_part * max(1, len(parts)))()
    keep = [arr]
    for k, q in enumerate(parts):  # composite grain (Sec. 4): discs and convex polygons in order
        arr[k].kind = PART_KINDS[q["kind"]]
        arr[k].add = 1 if q.get("add", True) else 0
        if q["kind"] == "disc":
            arr[k].cx, arr[k].cy, arr[k].r = float(q["cx"]), float(q["cy"]), float(q["r"])
        else:
            ax = np.ascontiguousarray(q["vx"], np.float64)
            ay = np.ascontiguousarray(q["vy"], np.float64)
            keep += [ax, ay]
            arr[k].n_vert = len(ax)
            arr[k].vx = ax.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            arr[k].vy = ay.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    p.n_parts = len(parts)
    p.parts = ctypes.cast(arr, ctypes.POINTER(sc_part))
    p.eps_cut = float(d.get("eps_cut", 0.0))
    p.adjoint_checkpoint = int(d.get("adjoint_checkpoint", 0))
    if d.get("mask") is not None:  # the caller's expectation of the grain mask, checked by sc_create
        mk = np.ascontiguousarray(d["mask"], np.uint8)
        keep.append(mk)
        p.mask = mk.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    p._keep = (vx, vy, keep)
    return p


def sc_create(params):
    h = ctypes.c_void_p()
    _check(lib.sc_create(ctypes.byref(params), ctypes.byref(h)))
    return h


def sc_destroy(ctx):
    _check(lib.sc_destroy(ctx))


def sc_get_info(ctx):
    i = sc_info()
    _check(lib.sc_get_info(ctx, ctypes.byref(i)), ctx)
    return i


def sc_set_fields(ctx, delta, a_ind=None, on_device=True, stream=None):
    _check(lib.sc_set_fields(ctx, _ptr(delta), _ptr(a_ind), int(on_device), _stream(stream)), ctx)


def sc_reset_boundary(ctx):
    _check(lib.sc_reset_boundary(ctx), ctx)


def sc_riccati_sweep(ctx, stream=None):
    _check(lib.sc_riccati_sweep(ctx, _stream(stream)), ctx)


def sc_burnin(ctx, max_sweeps, tol, stream=None):
    st = lib.sc_burnin(ctx, int(max_sweeps), float(tol), _stream(stream))
    if st not in (SC_OK, SC_ENOTCONV):
        _check(st, ctx)
    return st == SC_OK


def sc_gap_update(ctx, delta_out, on_device=True, want_eps=False, stream=None):
    eps = ctypes.c_double(0.0)
    _check(lib.sc_gap_update(ctx, _ptr(delta_out), ctypes.byref(eps) if want_eps else None,
                             int(on_device), _stream(stream)), ctx)
    return eps.value if want_eps else None


def sc_current(ctx, j_out, on_device=True, stream=None):
    _check(lib.sc_current(ctx, _ptr(j_out), int(on_device), _stream(stream)), ctx)


def sc_free_energy(ctx, density_out=None, on_device=True, want_total=True, stream=None):
    F = ctypes.c_double(0.0)
    _check(lib.sc_free_energy(ctx, ctypes.byref(F) if want_total else None, _ptr(density_out),
                              int(on_device), _stream(stream)), ctx)
    return F.value if want_total else None


def sc_update_vector_potential(ctx, stream=None):
    _check(lib.sc_update_vector_potential(ctx, _stream(stream)), ctx)


def sc_picard_step(ctx, stream=None):
    _check(lib.sc_picard_step(ctx, _stream(stream)), ctx)


def sc_ozaki_poles(n):
    """Ozaki's poles z (ascending) and residues R of the n-pole representation."""
    z, R = np.zeros(n), np.zeros(n)
    _check(lib.sc_ozaki_poles(int(n), _ptr(z), _ptr(R)))
    return z, R


def sc_ozaki_poles_for_cutoff(t, eps_cut):
    """The fewest Ozaki poles whose largest energy reaches eps_cut (0: none)."""
    return int(lib.sc_ozaki_poles_for_cutoff(ctypes.c_double(t), ctypes.c_double(eps_cut)))


def sc_debug_fp64_math(x, stream=None):
    """The sweep's FP64 device reciprocal and reciprocal square root of the
    device tensor x (float64): returns (1/x, 1/sqrt(x)) as device tensors."""
    import torch
    x = x.contiguous()
    rcp, rsq = torch.empty_like(x), torch.empty_like(x)
    _check(lib.sc_debug_fp64_math(_ptr(x), x.numel(), _ptr(rcp), _ptr(rsq), _stream(stream)))
    return rcp, rsq


def sc_debug_fma_rate(packed=True, stream=None):
    """Measured FP32 lane fused multiply-adds per second of this GPU."""
    r = ctypes.c_double(0.0)
    _check(lib.sc_debug_fma_rate(int(bool(packed)), ctypes.byref(r), _stream(stream)))
    return r.value


def sc_debug_validate_tables(ctx):
    """Number of out-of-range indices in the context's host tables."""
    n = ctypes.c_int64(0)
    _check(lib.sc_debug_validate_tables(ctx, ctypes.byref(n)), ctx)
    return n.value


def sc_debug_corrupt_table(ctx, which):
    """Make one host-table index of a host_only context out of range (tests)."""
    _check(lib.sc_debug_corrupt_table(ctx, int(which)), ctx)


def sc_debug_bounds(reset=False):
    """(violations, checked_build): index-check violations of the kernels on the
    current device and whether this library is the bounds-checked build."""
    v, c = ctypes.c_uint64(0), ctypes.c_int32(0)
    _check(lib.sc_debug_bounds(ctypes.byref(v), ctypes.byref(c), int(bool(reset))))
    return v.value, bool(c.value)


def sc_energy_grid(ctx, n_e):
    eps, w = np.zeros(n_e), np.zeros(n_e)
    _check(lib.sc_energy_grid(ctx, _ptr(eps), _ptr(w)), ctx)
    return eps, w


def sc_accel_params_default(kind):
    p = sc_accel_params()
    _check(lib.sc_accel_params_default(int(ACCELERATORS.get(kind, kind)), ctypes.byref(p)))
    return p


def accel_params(name, **overrides):
    """sc_accel_params with the paper's defaults for accelerator `name` and any
    overrides (fields of sc_accel_params)."""
    p = sc_accel_params_default(name)
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def sc_accelerate(ctx, params, stream=None):
    _check(lib.sc_accelerate(ctx, ctypes.byref(params), _stream(stream)), ctx)


def sc_accel_reset(ctx):
    _check(lib.sc_accel_reset(ctx), ctx)


def sc_get_history(ctx):
    """The context's residual records, oldest first: (sweeps run, eps_G) as two
    numpy arrays."""
    n = ctypes.c_int32(0)
    _check(lib.sc_get_history(ctx, ctypes.byref(n), None, None))
    cap = n.value
    sw = np.zeros(cap, dtype=np.int64)
    eps = np.zeros(cap, dtype=np.float64)
    if cap:
        n = ctypes.c_int32(cap)
        _check(lib.sc_get_history(ctx, ctypes.byref(n), sw.ctypes.data, eps.ctypes.data))
    return sw, eps


def sc_clear_history(ctx):
    _check(lib.sc_clear_history(ctx))


def sc_accel_get_state(ctx):
    """(iterations, step sizes, CongAcc weights): arrays of 2 n_components + 2
    entries (Re, Im of each Delta component, then A_x, A_y)."""
    it = ctypes.c_int32(0)
    a = np.zeros(10)
    w = np.zeros(10)
    _check(lib.sc_accel_get_state(ctx, ctypes.byref(it), _ptr(a), _ptr(w)), ctx)
    return it.value, a, w


def sc_ldos(ctx, energies, broadening, n_burnin, ldos_out, on_device=True, stream=None):
    e = np.ascontiguousarray(energies, np.float64)
    _check(lib.sc_ldos(ctx, _ptr(e), len(e), float(broadening), int(n_burnin), _ptr(ldos_out),
                       int(on_device), _stream(stream)), ctx)


def sc_sweep_lines_noalloc(samples, line_slot0, line_ns, line_len, entry, n_lines, max_ns, n_e,
                           t, h, images, exits, stream=None):
    """Allocation-free FP32 line sweep (no sc_ctx; every buffer is the
    caller's device memory; scratch is a static array inside the library).
    For callers that cannot allocate device memory at sweep time."""
    _check(lib.sc_sweep_lines_noalloc(_ptr(samples), _ptr(line_slot0), _ptr(line_ns), _ptr(line_len),
                                      _ptr(entry), int(n_lines), int(max_ns), int(n_e), float(t),
                                      float(h), _ptr(images), _ptr(exits), _stream(stream)))


def sc_sweep_adjoint(ctx, g_delta_new, g_j, g_F, g_Ftotal, dL_ddelta, dL_daind, on_device=True,
                     stream=None):
    _check(lib.sc_sweep_adjoint(ctx, _ptr(g_delta_new), _ptr(g_j), _ptr(g_F), float(g_Ftotal),
                                _ptr(dL_ddelta), _ptr(dL_daind), int(on_device), _stream(stream)), ctx)


def sc_ldos_adjoint(ctx, energies, broadening, n_burnin, g_ldos, dL_ddelta, dL_daind, on_device=True,
                    stream=None):
    e = np.ascontiguousarray(energies, np.float64)
    _check(lib.sc_ldos_adjoint(ctx, _ptr(e), len(e), float(broadening), int(n_burnin), _ptr(g_ldos),
                               _ptr(dL_ddelta), _ptr(dL_daind), int(on_device), _stream(stream)), ctx)


def sc_batch_create(params_list, energies_per_lane=0):
    arr = (sc_params * len(params_list))(*params_list)
    h = ctypes.c_void_p()
    _check(lib.sc_batch_create(arr, len(params_list), int(energies_per_lane), ctypes.byref(h)))
    return h


def sc_batch_destroy(b):
    _check(lib.sc_batch_destroy(b))


def sc_batch_member(b, i):
    h = ctypes.c_void_p()
    _check(lib.sc_batch_member(b, int(i), ctypes.byref(h)))
    return h


def sc_batch_sweep(b, stream=None):
    _check(lib.sc_batch_sweep(b, _stream(stream)))


def sc_batch_run(b, n_sweeps, with_outputs=True, stream=None):
    _check(lib.sc_batch_run(b, int(n_sweeps), int(bool(with_outputs)), _stream(stream)))


def sc_batch_set_energy_parts(b, on):
    """FP32: let padded members run their energies as two parts (layout rebuilt)."""
    _check(lib.sc_batch_set_energy_parts(b, int(bool(on))))


def sc_batch_set_fused_transfers(b, on):
    """FP32: run the members' rotations and rotate-backs as work items of the
    sweep's class launches (layout rebuilt)."""
    _check(lib.sc_batch_set_fused_transfers(b, int(bool(on))))


def sc_batch_reset_boundary(b):
    """The next batch sweep starts from fresh boundary values (layout kept)."""
    _check(lib.sc_batch_reset_boundary(b))


def sc_batch_autotune(b, stream=None):
    e = ctypes.c_int32(0)
    _check(lib.sc_batch_autotune(b, ctypes.byref(e), _stream(stream)))
    return e.value


def sc_batch_get_info(b):
    i = sc_batch_info()
    _check(lib.sc_batch_get_info(b, ctypes.byref(i)))
    return i


def sc_batch_set_fields(b, delta_all, on_device=True, stream=None):
    """Every member's Delta from one array (members one after another)."""
    _check(lib.sc_batch_set_fields(b, _ptr(delta_all), int(on_device), _stream(stream)))


def sc_batch_get_outputs(b, delta_new_all=None, j_all=None, F_all=None, on_device=True, stream=None):
    """Every member's Delta_new, j, F into arrays of all members (any may be None)."""
    _check(lib.sc_batch_get_outputs(b, _ptr(delta_new_all), _ptr(j_all), _ptr(F_all), int(on_device),
                                    _stream(stream)))


class Batch:
    """Many grains swept by one persistent launch."""

    def __init__(self, prms, precision="fp32", energies_per_lane=0):
        self.prms = [dict(p) for p in prms]
        self._p = [make_params(p, precision) for p in prms]
        self.h = sc_batch_create(self._p, energies_per_lane)
        self.members = []
        for i, p in enumerate(prms):
            m = Context.__new__(Context)
            m.prm = dict(p)
            m._p = self._p[i]
            m.h = sc_batch_member(self.h, i)
            m.info = sc_get_info(m.h)
            m.nx, m.ny, m.n_e, m.N = p["nx"], p["ny"], p["n_energies"], p["n_angles"]
            m._owned = False
            self.members.append(m)

    def sweep(self, stream=None):
        sc_batch_sweep(self.h, stream)

    def autotune(self, stream=None):
        return sc_batch_autotune(self.h, stream)

    def run(self, n_sweeps, with_outputs=True, stream=None):
        sc_batch_run(self.h, n_sweeps, with_outputs, stream)

    def reset_boundary(self):
        sc_batch_reset_boundary(self.h)

    def set_fused_transfers(self, on):
        sc_batch_set_fused_transfers(self.h, on)

    def info(self):
        return sc_batch_get_info(self.h)

    def close(self):
        if self.h:
            for m in self.members:
                m.h = None
            sc_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context:
    """One grain: owns an sc_ctx.  Arrays in, arrays out (torch on the GPU)."""

    def __init__(self, prm, precision="fp32", lanes_per_line=0, host_only=False,
                 record_timings=False):
        self.prm = dict(prm)
        self._p = make_params(prm, precision, lanes_per_line, host_only, record_timings)
        self.h = sc_create(self._p)
        self.info = sc_get_info(self.h)
        self.nx, self.ny = prm["nx"], prm["ny"]
        self.n_e = prm["n_energies"]
        self.N = prm["n_angles"]
        self.sweep_count = 0

    def close(self):
        if self.h and getattr(self, "_owned", True):
            sc_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- geometry (host) --------------------------------------------------
    def mask(self):
        m = np.zeros((self.ny, self.nx), np.uint8)
        _check(lib.sc_get_mask(self.h, _ptr(m)), self.h)
        return m

    def lines(self):
        P, L = self.info.n_pairs, self.info.n_lines
        lo, hi = np.zeros(P, np.int32), np.zeros(P, np.int32)
        smin, smax = np.zeros(L), np.zeros(L)
        m0, m1 = np.zeros(L, np.int32), np.zeros(L, np.int32)
        _check(lib.sc_debug_lines(self.h, _ptr(lo), _ptr(hi), _ptr(smin), _ptr(smax), _ptr(m0),
                                  _ptr(m1)), self.h)
        pair, l = np.zeros(L, np.int32), np.zeros(L, np.int32)
        _check(lib.sc_debug_chords(self.h, _ptr(pair), _ptr(l)), self.h)
        return dict(l_lo=lo, l_hi=hi, smin=smin, smax=smax, m0=m0, m1=m1, pair=pair, l=l)

    def ghost(self):
        g = np.zeros((self.ny + 2, self.nx + 2), np.int32)
        _check(lib.sc_debug_ghost(self.h, _ptr(g)), self.h)
        return g

    def links(self):
        n = 4 * 2 * self.info.n_lines
        ta, tl, tc, tw = np.zeros(n, np.int32), np.zeros(n, np.int32), np.zeros(n, np.int32), np.zeros(n)
        _check(lib.sc_debug_links(self.h, _ptr(ta), _ptr(tl), _ptr(tc), _ptr(tw)), self.h)
        return dict(angle=ta.reshape(-1, 4), line=tl.reshape(-1, 4), chord=tc.reshape(-1, 4),
                    w=tw.reshape(-1, 4))

    # -- compute (device) -------------------------------------------------
    def set_fields(self, delta, aind=None, stream=None):
        import torch
        d = torch.view_as_real(torch.as_tensor(delta, dtype=torch.complex128, device="cuda").contiguous()).contiguous()
        a = None
        if aind is not None:
            a = torch.as_tensor(aind, dtype=torch.float64, device="cuda").contiguous()
        self._fields = (d, a)  # keep alive until the copy ran
        sc_set_fields(self.h, d, a, True, stream)

    def fields(self, stream=None):
        """The context's current Delta (complex, (ny, nx) or (C, ny, nx)) and
        A_ind ((ny, nx, 2)) as device tensors."""
        import torch
        d = torch.empty(self._dshape() + (2,), dtype=torch.float64, device="cuda")
        a = torch.empty((self.prm["ny"], self.prm["nx"], 2), dtype=torch.float64, device="cuda")
        _check(lib.sc_get_fields(self.h, _ptr(d), _ptr(a), 1, _stream(stream)), self.h)
        return torch.view_as_complex(d), a

    def sweep(self, stream=None):
        sc_riccati_sweep(self.h, stream)
        self.sweep_count = getattr(self, "sweep_count", 0) + 1

    @property
    def n_comp(self):
        return max(1, len(self.prm.get("components") or []))

    def _dshape(self):
        """Shape of Delta-like complex fields: (ny, nx), or (C, ny, nx) with C > 1 components."""
        return (self.n_comp, self.ny, self.nx) if self.n_comp > 1 else (self.ny, self.nx)

    def outputs(self, stream=None):
        import torch
        dn = torch.empty(self._dshape() + (2,), dtype=torch.float64, device="cuda")
        j = torch.empty((self.ny, self.nx, 2), dtype=torch.float64, device="cuda")
        F = torch.empty((self.ny, self.nx), dtype=torch.float64, device="cuda")
        eps = sc_gap_update(self.h, dn, True, True, stream)
        sc_current(self.h, j, True, stream)
        Ft = sc_free_energy(self.h, F, True, True, stream)
        return dict(delta_new=torch.view_as_complex(dn), j=j, F=F, F_total=Ft, eps_G=eps)

    def exits(self):
        out = np.zeros(2 * 2 * self.info.n_lines * self.n_e)
        _check(lib.sc_debug_exits(self.h, _ptr(out)), self.h)
        return out.view(np.complex128).reshape(2 * self.info.n_lines, self.n_e)

    def images(self):
        out = np.zeros(4 * self.info.n_samples)
        _check(lib.sc_debug_images(self.h, _ptr(out)), self.h)
        return out.reshape(-1, 4)

    def adjoint(self, g_delta_new=None, g_j=None, g_F=None, g_Ftotal=0.0, stream=None):
        """dL/dDelta(R) (complex) and dL/dA_ind(R) for output cotangents of the
        last sweep (torch tensors or arrays; None = zero)."""
        import torch

        def dev(x, shape_last):
            if x is None:
                return None
            t = torch.as_tensor(x, device="cuda")
            if t.is_complex():
                t = torch.view_as_real(t.to(torch.complex128).contiguous())
            return t.to(torch.float64).contiguous()
        gdn, gj, gF = dev(g_delta_new, 2), dev(g_j, 2), dev(g_F, 1)
        dd = torch.empty(self._dshape() + (2,), dtype=torch.float64, device="cuda")
        da = torch.empty((self.ny, self.nx, 2), dtype=torch.float64, device="cuda")
        sc_sweep_adjoint(self.h, gdn, gj, gF, g_Ftotal, dd, da, True, stream)
        self._adj_keep = (gdn, gj, gF)
        return torch.view_as_complex(dd), da

    def ldos_adjoint(self, energies, broadening, g_ldos, n_burnin=20, stream=None):
        """dL/dDelta(R) (complex) and dL/dA_ind(R) for an LDOS-map cotangent g_ldos
        (n_e x ny x nx)."""
        import torch
        g = torch.as_tensor(g_ldos, dtype=torch.float64, device="cuda").contiguous()
        dd = torch.empty(self._dshape() + (2,), dtype=torch.float64, device="cuda")
        da = torch.empty((self.ny, self.nx, 2), dtype=torch.float64, device="cuda")
        sc_ldos_adjoint(self.h, energies, broadening, n_burnin, g, dd, da, True, stream)
        return torch.view_as_complex(dd), da

    def accelerate(self, params, stream=None):
        """One accelerator step (App. E) after a sweep: params from accel_params()."""
        sc_accelerate(self.h, params, stream)

    def self_consistency(self, params, max_iter=1000, tol=1e-5, check_every=1, stream=None):
        """The native loop of Algorithm 1 (sweep, residual check, accelerator
        step): returns (converged, iterations, eps_G)."""
        it = ctypes.c_int32(0)
        eps = ctypes.c_double(0.0)
        st = lib.sc_self_consistency(self.h, ctypes.byref(params), int(max_iter), float(tol), int(check_every),
                                     ctypes.byref(it), ctypes.byref(eps), _stream(stream))
        if st not in (SC_OK, SC_ENOTCONV):
            _check(st, self.h)
        return st == SC_OK, it.value, eps.value

    def history(self):
        """Residual records of this context, oldest first: (sweeps, eps_G)."""
        return sc_get_history(self.h)

    def clear_history(self):
        sc_clear_history(self.h)

    def ldos(self, energies, broadening, n_burnin=20, stream=None):
        import torch
        out = torch.empty((len(energies), self.ny, self.nx), dtype=torch.float64, device="cuda")
        sc_ldos(self.h, energies, broadening, n_burnin, out, True, stream)
        return out
