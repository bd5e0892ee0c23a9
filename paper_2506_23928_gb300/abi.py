"""ctypes binding of libotvmc (include/otvmc.h): the same entry points, argument marshalling only.

Every function takes torch tensors (device or host, as the C signature says), Python ints
(raw pointers) or None, and returns the otvmc_status code; `check(status)` raises on error.
Loading fails loudly when the library has not been built: there is no fallback path.
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libotvmc.so")

OTVMC_OK = 0
OTVMC_ERR_INVALID = 1
OTVMC_ERR_OOM = 2
OTVMC_ERR_CUDA = 3
OTVMC_ERR_NOT_PD = 4
OTVMC_ERR_TIMEOUT = 5
OTVMC_ERR_NONFINITE = 6
OTVMC_ERR_RANGE = 7
OTVMC_ERR_UNSUPPORTED = 8
OTVMC_ERR_WORKSPACE = 9
OTVMC_JASTROW, OTVMC_RBM, OTVMC_LJ = 0, 1, 2
OTVMC_PREC_FP64, OTVMC_PREC_MIXED = 0, 1
OTVMC_REG_SHIFT, OTVMC_REG_SNR = 0, 1
OTVMC_HEUN, OTVMC_MIDPOINT = 0, 1
OTVMC_RBM_T_FACTORED, OTVMC_RBM_T_MATERIALISED = 0, 1
OTVMC_PROFILE_OFF, OTVMC_PROFILE_ON, OTVMC_PROFILE_SERIAL = 0, 1, 2
OTVMC_MOMENTS = 9
OTVMC_MAX_GROUPS = 8
KERNEL_CLASSES = ["sample", "prep", "est1", "est2", "reduce", "obs", "D", "obuild", "gram", "syrk", "solve", "sde",
                  "noise", "chol_update", "chol_trsm", "chol_diag", "chol_resid"]

c_int, c_int64, c_uint64, c_double, c_size_t, c_void_p = (ctypes.c_int, ctypes.c_int64, ctypes.c_uint64,
                                                         ctypes.c_double, ctypes.c_size_t, ctypes.c_void_p)


class ModelDesc(ctypes.Structure):
    _fields_ = [("n", c_int), ("J_h", c_void_p), ("h", c_double), ("kappa_h", c_void_p), ("gamma_h", c_void_p)]


class RunDesc(ctypes.Structure):
    _fields_ = [("ntraj", c_int), ("traj0", c_int), ("ns", c_int), ("n_steps", c_int), ("step0", c_int64),
                ("n_sweep", c_int), ("dt", c_double), ("scheme", c_int), ("precision", c_int), ("reg", c_int),
                ("eps", c_double), ("snr_thresh", c_double), ("seed", c_uint64), ("measure_every", c_int),
                ("measure_final", c_int), ("use_graph", c_int)]


# name -> (restype, argtypes); pointers are passed as c_void_p
P = c_void_p
SIGNATURES = {
    "otvmc_lattice_couplings": (c_int, [c_int, P, c_double, c_double, c_int, c_int, P]),
    "otvmc_model_create": (c_int, [P, P]),
    "otvmc_model_destroy": (None, [P]),
    "otvmc_model_nops": (c_int, [P]),
    "otvmc_ansatz_create": (c_int, [P, c_int, c_int, P]),
    "otvmc_ansatz_create_lj": (c_int, [P, c_int, c_int, P]),
    "otvmc_ansatz_destroy": (None, [P]),
    "otvmc_ansatz_nparams": (c_int64, [P]),
    "otvmc_ansatz_set_rbm_t_build": (c_int, [P, c_int]),
    "otvmc_workspace_bytes": (c_size_t, [P, c_int, c_int, c_int]),
    "otvmc_check": (c_int, [P, P]),
    "otvmc_draw_noise": (c_int, [P, c_int, c_int, c_uint64, c_int64, c_double, P, P]),
    "otvmc_init_chains": (c_int, [P, c_int, c_int, c_int, c_uint64, P, P]),
    "otvmc_sample": (c_int, [P, P, c_int, c_int, c_int, c_int, c_uint64, c_int64, P, P, P, c_size_t, P]),
    "otvmc_local_estimators": (c_int, [P, P, P, c_int, c_int, P, c_double, c_int, P, P, P, P, c_size_t, P]),
    "otvmc_local_estimators_noalloc": (c_int, [P, P, P, c_int, c_int, P, c_double, c_int, P, P, P, P, P]),
    "otvmc_build_S_F": (c_int, [P, P, P, P, c_int, c_int, c_int, P, P, P, P, P, c_size_t, P]),
    "otvmc_solve_step": (c_int, [P, c_int, c_int, c_int, c_int, c_double, c_double, P, P, P, P, P, P, P, c_size_t,
                                 P]),
    "otvmc_solve_snr": (c_int, [P, c_int, c_int, P, P, P, P, P, c_double, c_double, P, P, P, c_size_t, P]),
    "otvmc_snr_workspace_bytes": (c_size_t, [P, c_int]),
    "otvmc_sde_combine": (c_int, [c_int, c_int64, c_int, c_int, P, P, P, P, P, P, c_size_t, P]),
    "otvmc_observables": (c_int, [P, P, P, c_int, c_int, c_int, P, P, c_size_t, P]),
    "otvmc_ensemble": (c_int, [P, c_int, c_int, P, P, P, P]),
    "otvmc_run_workspace_bytes": (c_size_t, [P, P]),
    "otvmc_run_n_meas": (c_int, [P]),
    "otvmc_run_trajectories": (c_int, [P, P, P, P, P, P, c_size_t, P]),
    "otvmc_run_trajectories_linear": (c_int, [P, P, P, P, P, P, P, P, c_size_t, P]),
    "otvmc_run_grouped_workspace_bytes": (c_size_t, [P, P, c_int]),
    "otvmc_autotune_workspace_bytes": (c_size_t, [P, P]),
    "otvmc_autotune_run": (c_int, [P, P, P, P, P, c_size_t, P, P, P, P]),
    "otvmc_autotune_clear": (None, []),
    "otvmc_run_trajectories_grouped": (c_int, [P, P, c_int, P, P, P, P, c_size_t, P]),
    "otvmc_ensemble_weighted": (c_int, [P, P, c_int, c_int, P, P, P, P]),
    "otvmc_run_host_workspace_bytes": (c_size_t, [P, P]),
    "otvmc_run_trajectories_host": (c_int, [P, P, P, P, P, P, c_size_t, P]),
    "otvmc_profile_enable": (None, [c_int]),
    "otvmc_profile_read": (c_int, [c_int, P, P]),
    "otvmc_last_error": (ctypes.c_char_p, []),
    "otvmc_launch_count": (c_uint64, []),
    "otvmc_debug_set_wait_limit": (c_int, [c_uint64]),
}

_lib = None


def load():
    """Loads libotvmc.so (built by paper_2506_23928_gb300.build); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libotvmc.so not built ({LIB_PATH}); run paper_2506_23928_gb300.build.build()")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def ptr(x):
    """Raw address of a torch tensor / numpy array / ctypes object / int, or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    return ctypes.addressof(x)


def stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class OtvmcError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"otvmc status {status}: {msg}")
        self.status = status


def check(status):
    if status != OTVMC_OK:
        raise OtvmcError(status, load().otvmc_last_error().decode())
    return status


def _call(name, *args):
    return getattr(load(), name)(*args)


def otvmc_lattice_couplings(dim, extent, J, alpha, kac, pbc, J_out_h):
    ext = (ctypes.c_int * len(extent))(*extent)
    return _call("otvmc_lattice_couplings", dim, ctypes.addressof(ext), J, alpha, int(kac), int(pbc), ptr(J_out_h))


def otvmc_model_create(desc, out):
    return _call("otvmc_model_create", ctypes.addressof(desc), ctypes.addressof(out))


def otvmc_model_destroy(model):
    _call("otvmc_model_destroy", model)


def otvmc_model_nops(model):
    return _call("otvmc_model_nops", model)


def otvmc_ansatz_create(model, kind, n_hidden, out):
    return _call("otvmc_ansatz_create", model, kind, n_hidden, ctypes.addressof(out))


def otvmc_ansatz_create_lj(model, d, pbc, out):
    return _call("otvmc_ansatz_create_lj", model, d, pbc, ctypes.addressof(out))


def otvmc_ansatz_destroy(ansatz):
    _call("otvmc_ansatz_destroy", ansatz)


def otvmc_ansatz_nparams(ansatz):
    return _call("otvmc_ansatz_nparams", ansatz)


def otvmc_ansatz_set_rbm_t_build(ansatz, mode):
    return _call("otvmc_ansatz_set_rbm_t_build", ansatz, mode)


def otvmc_workspace_bytes(ansatz, ntraj, ns, precision):
    return _call("otvmc_workspace_bytes", ansatz, ntraj, ns, precision)


def otvmc_check(work_d, stream=None):
    return _call("otvmc_check", ptr(work_d), stream_ptr(stream))


def otvmc_draw_noise(model, ntraj, traj0, seed, step, dt, dW_d, stream=None):
    return _call("otvmc_draw_noise", model, ntraj, traj0, seed, step, dt, ptr(dW_d), stream_ptr(stream))


def otvmc_init_chains(ansatz, ntraj, traj0, ns, seed, spins_d, stream=None):
    return _call("otvmc_init_chains", ansatz, ntraj, traj0, ns, seed, ptr(spins_d), stream_ptr(stream))


def otvmc_sample(ansatz, theta_d, ntraj, traj0, ns, n_sweep, seed, eval_index, spins_d, accepted_d, work_d,
                 work_bytes, stream=None):
    return _call("otvmc_sample", ansatz, ptr(theta_d), ntraj, traj0, ns, n_sweep, seed, eval_index, ptr(spins_d),
                 ptr(accepted_d), ptr(work_d), work_bytes, stream_ptr(stream))


def otvmc_local_estimators(ansatz, theta_d, spins_d, ntraj, ns, dW_d, dt, precision, Eeff_d, v_d, lpl_d, work_d,
                           work_bytes, stream=None):
    return _call("otvmc_local_estimators", ansatz, ptr(theta_d), ptr(spins_d), ntraj, ns, ptr(dW_d), dt, precision,
                 ptr(Eeff_d), ptr(v_d), ptr(lpl_d), ptr(work_d), work_bytes, stream_ptr(stream))


def otvmc_local_estimators_noalloc(ansatz, theta_d, spins_d, ntraj, ns, dW_d, dt, precision, Eeff_d, v_d, lpl_d,
                                   status_d, stream=None):
    return _call("otvmc_local_estimators_noalloc", ansatz, ptr(theta_d), ptr(spins_d), ntraj, ns, ptr(dW_d), dt,
                 precision, ptr(Eeff_d), ptr(v_d), ptr(lpl_d), ptr(status_d), stream_ptr(stream))


def otvmc_build_S_F(ansatz, theta_d, spins_d, v_d, ntraj, ns, precision, S_d, G_d, obar_d, D_d, work_d, work_bytes,
                    stream=None):
    return _call("otvmc_build_S_F", ansatz, ptr(theta_d), ptr(spins_d), ptr(v_d), ntraj, ns, precision, ptr(S_d),
                 ptr(G_d), ptr(obar_d), ptr(D_d), ptr(work_d), work_bytes, stream_ptr(stream))


def otvmc_solve_step(ansatz, ntraj, ns, precision, reg, eps, snr_thresh, S_d, G_d, obar_d, D_d, delta_d,
                     shift_used_d, work_d, work_bytes, stream=None):
    return _call("otvmc_solve_step", ansatz, ntraj, ns, precision, reg, eps, snr_thresh, ptr(S_d), ptr(G_d),
                 ptr(obar_d), ptr(D_d), ptr(delta_d), ptr(shift_used_d), ptr(work_d), work_bytes, stream_ptr(stream))


def otvmc_solve_snr(ansatz, ntraj, ns, S_d, obar_d, spins_d, v_d, D_d, snr_thresh, eps_svd, delta_d, lambda_d,
                    work_d, work_bytes, stream=None):
    return _call("otvmc_solve_snr", ansatz, ntraj, ns, ptr(S_d), ptr(obar_d), ptr(spins_d), ptr(v_d), ptr(D_d),
                 snr_thresh, eps_svd, ptr(delta_d), ptr(lambda_d), ptr(work_d), work_bytes, stream_ptr(stream))


def otvmc_sde_combine(ntraj, P_, scheme, stage, theta_d, delta0_d, delta1_d, out_d, failed_d, work_d, work_bytes,
                      stream=None):
    return _call("otvmc_sde_combine", ntraj, P_, scheme, stage, ptr(theta_d), ptr(delta0_d), ptr(delta1_d),
                 ptr(out_d), ptr(failed_d), ptr(work_d), work_bytes, stream_ptr(stream))


def otvmc_observables(ansatz, theta_d, spins_d, ntraj, ns, precision, moments_d, work_d, work_bytes, stream=None):
    return _call("otvmc_observables", ansatz, ptr(theta_d), ptr(spins_d), ntraj, ns, precision, ptr(moments_d),
                 ptr(work_d), work_bytes, stream_ptr(stream))


def otvmc_ensemble(moments_h, ntraj, n_sites, M_h, C_h, xi2_h, dM_h):
    return _call("otvmc_ensemble", ptr(moments_h), ntraj, n_sites, ptr(M_h), ptr(C_h), ptr(xi2_h), ptr(dM_h))


def otvmc_run_workspace_bytes(ansatz, desc):
    return _call("otvmc_run_workspace_bytes", ansatz, ctypes.addressof(desc))


def otvmc_run_n_meas(desc):
    return _call("otvmc_run_n_meas", ctypes.addressof(desc))


def otvmc_run_trajectories(ansatz, desc, theta_d, spins_d, moments_d, work_d, work_bytes, stream=None):
    return _call("otvmc_run_trajectories", ansatz, ctypes.addressof(desc), ptr(theta_d), ptr(spins_d),
                 ptr(moments_d), ptr(work_d), work_bytes, stream_ptr(stream))


def _desc_array(descs):
    arr = (RunDesc * len(descs))()
    for i, d in enumerate(descs):
        arr[i] = d
    return arr


def otvmc_autotune_workspace_bytes(ansatz, desc):
    return _call("otvmc_autotune_workspace_bytes", ansatz, ctypes.addressof(desc))


def otvmc_autotune_run(ansatz, desc, theta_d, spins_d, work_d, work_bytes, stream=None):
    """Returns (status, sub-batches, solver groups, ms per step) of the recorded shape."""
    pipes, groups, ms = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_double(0.0)
    st = _call("otvmc_autotune_run", ansatz, ctypes.addressof(desc), ptr(theta_d), ptr(spins_d), ptr(work_d),
               work_bytes, stream_ptr(stream), ctypes.addressof(pipes), ctypes.addressof(groups),
               ctypes.addressof(ms))
    return st, pipes.value, groups.value, ms.value


def otvmc_autotune_clear():
    _call("otvmc_autotune_clear")


def otvmc_snr_workspace_bytes(ansatz, ntraj):
    return _call("otvmc_snr_workspace_bytes", ansatz, ntraj)


def otvmc_run_grouped_workspace_bytes(ansatz, descs):
    arr = _desc_array(descs)
    return _call("otvmc_run_grouped_workspace_bytes", ansatz, ctypes.addressof(arr), len(descs))


def otvmc_run_trajectories_grouped(ansatz, descs, thetas, spins, moments, work_d, work_bytes, stream=None):
    """descs, thetas, spins, moments: one entry per group (moments entries may be None)."""
    n = len(descs)
    arr = _desc_array(descs)
    th = (ctypes.c_void_p * n)(*[ptr(x) for x in thetas])
    sp = (ctypes.c_void_p * n)(*[ptr(x) for x in spins])
    mo = (ctypes.c_void_p * n)(*[ptr(x) for x in moments])
    return _call("otvmc_run_trajectories_grouped", ansatz, ctypes.addressof(arr), n, ctypes.addressof(th),
                 ctypes.addressof(sp), ctypes.addressof(mo), ptr(work_d), work_bytes, stream_ptr(stream))


def otvmc_run_trajectories_linear(ansatz, desc, theta_d, spins_d, moments_d, lnQ_d, lnQ_rows_d, work_d, work_bytes,
                                  stream=None):
    return _call("otvmc_run_trajectories_linear", ansatz, ctypes.addressof(desc), ptr(theta_d), ptr(spins_d),
                 ptr(moments_d), ptr(lnQ_d), ptr(lnQ_rows_d), ptr(work_d), work_bytes, stream_ptr(stream))


def otvmc_ensemble_weighted(moments_h, w_h, ntraj, n_sites, M_h, C_h, xi2_h, dM_h):
    return _call("otvmc_ensemble_weighted", ptr(moments_h), ptr(w_h), ntraj, n_sites, ptr(M_h), ptr(C_h), ptr(xi2_h),
                 ptr(dM_h))


def otvmc_run_host_workspace_bytes(ansatz, desc):
    return _call("otvmc_run_host_workspace_bytes", ansatz, ctypes.addressof(desc))


def otvmc_run_trajectories_host(ansatz, desc, theta_h, spins_h, moments_h, work_d, work_bytes, stream=None):
    return _call("otvmc_run_trajectories_host", ansatz, ctypes.addressof(desc), ptr(theta_h), ptr(spins_h),
                 ptr(moments_h), ptr(work_d), work_bytes, stream_ptr(stream))


def otvmc_profile_enable(on):
    _call("otvmc_profile_enable", int(on))


def otvmc_profile_read(kernel_class, total_ms, launches):
    return _call("otvmc_profile_read", kernel_class, ctypes.addressof(total_ms), ctypes.addressof(launches))


def profile_summary():
    """{class name: (total ms, launches)} of the kernels recorded since profiling was enabled."""
    out = {}
    for i, name in enumerate(KERNEL_CLASSES):
        ms, cnt = ctypes.c_double(), ctypes.c_uint64()
        check(otvmc_profile_read(i, ms, cnt))
        if cnt.value:
            out[name] = (ms.value, cnt.value)
    return out


def otvmc_last_error():
    return _call("otvmc_last_error").decode()


def otvmc_launch_count():
    return _call("otvmc_launch_count")


def otvmc_debug_set_wait_limit(ns):
    return _call("otvmc_debug_set_wait_limit", ns)
