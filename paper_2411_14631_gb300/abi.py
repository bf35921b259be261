"""ctypes view of include/amrhydro.h and loader of the in-tree libamrhydro.so.

Argument marshalling only: every computation runs in the library's CUDA kernels.
Loading fails loudly if the library is missing; there is no other implementation."""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libamrhydro.so")
MAXLEV = 21
NCOUNTERS = 8

OK, EINVAL, EUNBALANCED, ECAPACITY, ECUDA, ETIMEOUT, ENONPHYSICAL, ENOCONV, EBREAKDOWN = 0, -1, -2, -3, -4, -5, -6, -7, -8
BC_PERIODIC, BC_OUTFLOW = 0, 1
RIEMANN_HLLC, RIEMANN_EXACT, RIEMANN_MLP, RIEMANN_MLP_SEEDED = 0, 1, 2, 3
PREC_FP64, PREC_FP32 = 0, 1
LIMITER_MINMOD, LIMITER_MC = 0, 1
PRECOND_NONE, PRECOND_IP = 0, 1
OP_A, OP_MINV = 0, 1

EXPORTS = ["amr_build_octree_query", "amr_build_octree", "hydro_init_from_prim", "hydro_prim_of_state",
           "hydro_courant", "hydro_godunov_level", "hydro_flux_reg_bytes", "hydro_reflux_level", "reflux_level", "hydro_step",
           "amr_get_status", "amr_status_string", "hydro_step_static_scratch", "hydro_harvest_faces",
           "mlp_nparams", "mlp_packed_bytes", "mlp_scratch_bytes", "mlp_pack", "mlp_make_dataset", "mlp_forward",
           "mlp_forward_tc", "mlp_tanh_rate",
           "mlp_grad", "mlp_train_step",
           "ppcg_workspace_bytes", "poisson_apply", "ppcg_start", "ppcg_iterate", "ppcg_poll", "ppcg_solve",
           "amr_refine_work_bytes", "amr_refine", "amr_build_octree_device_query", "amr_build_octree_device",
           "amr_remap_state", "hydro_courant_levels", "hydro_step_subcycled", "hydro_state_to_fp32",
           "hydro_state_from_fp32", "hydro_conservation_work_bytes", "hydro_conservation", "hydro_restrict_complete"]
MLP_NPARAMS = 8962
STATIC_REG_MAX_OCTS = 131072


class AmrGeom(C.Structure):
    _fields_ = [("levelmin", C.c_int32), ("bc", C.c_int32 * 6), ("n_inst", C.c_int32), ("h_inst_n", C.c_void_p)]


class HydroParams(C.Structure):
    _fields_ = [("gamma", C.c_double), ("cfl", C.c_double), ("rho_floor", C.c_double), ("p_floor", C.c_double),
                ("riemann", C.c_int32), ("precision", C.c_int32), ("tile", C.c_int32), ("tiles_only", C.c_int32),
                ("mlp_weights", C.c_void_p), ("mlp_resid_tol", C.c_float), ("limiter", C.c_int32),
                ("d_status", C.c_void_p), ("d_counters", C.c_void_p), ("col_kernel", C.c_int32),
                ("col_seg", C.c_int32), ("defer_restriction", C.c_int32), ("reserved", C.c_int32)]


class AmrTree(C.Structure):
    _fields_ = [("noct", C.c_int64), ("levelmin", C.c_int32), ("levelmax", C.c_int32), ("bc", C.c_int32 * 6),
                ("lvl_off", C.c_int64 * (MAXLEV + 2)), ("tile_off", (C.c_int64 * (MAXLEV + 2)) * 2),
                ("reg_base", C.c_int64),
                ("lvl", C.c_void_p), ("ix", C.c_void_p), ("iy", C.c_void_p), ("iz", C.c_void_p),
                ("key", C.c_void_p), ("son", C.c_void_p), ("father", C.c_void_p), ("nbor", C.c_void_p),
                ("nb27", C.c_void_p), ("refmask", C.c_void_p), ("fused", C.c_void_p),
                ("tile_root", C.c_void_p * 2),
                ("tile_slot", C.c_void_p * 2), ("n_inst", C.c_int32), ("inst_n", C.c_void_p), ("inst_dx", C.c_void_p),
                ("inst_oct_off", C.c_void_p), ("tile_inst", C.c_void_p * 2), ("grid_level", C.c_int32),
                ("grid", C.c_void_p), ("col_work", C.c_int64), ("inst_col_off", C.c_void_p),
                ("n_ghost", C.c_int64), ("ghost_off", C.c_int64 * (MAXLEV + 2)), ("ghost_cell", C.c_void_p),
                ("reflux_cell", C.c_void_p), ("reflux_off", C.c_int64 * (MAXLEV + 2))]


class RefineParams(C.Structure):
    _fields_ = [("mass_thr", C.c_double), ("levelmax", C.c_int32), ("pad", C.c_int32)]


class PpcgParams(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("precond", C.c_int32),
                ("tol", C.c_double), ("max_iter", C.c_int32), ("check_every", C.c_int32), ("tile_y", C.c_int32),
                ("seg", C.c_int32)]


class PpcgInfo(C.Structure):
    _fields_ = [("iters", C.c_int32), ("done", C.c_int32), ("status", C.c_int32), ("pad", C.c_int32),
                ("eps", C.c_double)]


_lib = None


def lib():
    """Load libamrhydro.so (built by ``paper_2411_14631_gb300.build``); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libamrhydro.so is not built (run paper_2411_14631_gb300.build.build()); "
                           "the hydro path has no other implementation")
    L = C.CDLL(LIB_PATH)
    P, S = C.c_void_p, C.c_size_t
    PT, PP = C.POINTER(AmrTree), C.POINTER(HydroParams)
    L.amr_build_octree_query.argtypes = [C.POINTER(AmrGeom), P, C.c_int64, C.POINTER(S), C.POINTER(S)]
    L.amr_build_octree.argtypes = [C.POINTER(AmrGeom), P, C.c_int64, P, S, P, S, PT, P]
    L.hydro_init_from_prim.argtypes = [PT, PP, P, P, P]
    L.hydro_prim_of_state.argtypes = [PT, PP, P, P, P]
    L.hydro_courant.argtypes = [PT, PP, P, P, P]
    L.hydro_godunov_level.argtypes = [PT, C.c_int, PP, P, P, P, P, P, P]
    L.hydro_flux_reg_bytes.argtypes = [PT]
    L.hydro_flux_reg_bytes.restype = S
    L.hydro_reflux_level.argtypes = [PT, C.c_int, PP, P, P, P, P, P]
    L.reflux_level.argtypes = [PT, C.c_int, PP, P, P, P, P, P]
    L.hydro_step.argtypes = [PT, PP, P, P, P, P, P, P]
    L.hydro_step_static_scratch.argtypes = [PT, PP, P, P, P, P, P]
    L.hydro_harvest_faces.argtypes = [PT, PP, P, P, P, C.c_int64, C.c_int64, P, P]
    L.mlp_nparams.argtypes = []
    L.mlp_packed_bytes.argtypes = []
    L.mlp_packed_bytes.restype = S
    L.mlp_scratch_bytes.argtypes = [C.c_int64]
    L.mlp_scratch_bytes.restype = S
    L.mlp_pack.argtypes = [P, P, P]
    L.mlp_make_dataset.argtypes = [P, C.c_int64, C.c_double, P, P, P, P]
    L.mlp_forward.argtypes = [P, P, P, C.c_int64, P]
    L.mlp_forward_tc.argtypes = [P, P, P, C.c_int64, P, P]
    L.mlp_tanh_rate.argtypes = [P, C.POINTER(C.c_int64), P]
    L.mlp_grad.argtypes = [P, P, P, C.c_int64, P, P, S, P]
    L.mlp_train_step.argtypes = [P, P, P, P, P, P, C.c_int64, C.c_float, C.c_int64, P, P, S, P]
    L.hydro_courant_levels.argtypes = [PT, PP, P, P, P]
    L.hydro_step_subcycled.argtypes = [PT, PP, P, P, P, P, P, P]
    L.amr_refine_work_bytes.argtypes = [PT]
    L.amr_refine_work_bytes.restype = S
    L.amr_refine.argtypes = [PT, C.POINTER(RefineParams), P, P, S, P, C.c_int64, P, C.POINTER(C.c_int64), P]
    L.amr_build_octree_device_query.argtypes = [C.POINTER(AmrGeom), P, C.POINTER(S), C.POINTER(S)]
    L.amr_build_octree_device.argtypes = [C.POINTER(AmrGeom), P, P, P, S, P, S, PT, P]
    L.amr_remap_state.argtypes = [PT, P, PT, P, P, P]
    PG = C.POINTER(PpcgParams)
    I = C.c_int32
    L.ppcg_workspace_bytes.argtypes = [I, I, I]
    L.ppcg_workspace_bytes.restype = S
    L.poisson_apply.argtypes = [I, I, I, I, P, P, P]
    L.ppcg_start.argtypes = [PG, P, P, P, S, P, P]
    L.ppcg_iterate.argtypes = [PG, P, P, S, P, I, P]
    L.ppcg_poll.argtypes = [P, C.POINTER(PpcgInfo), P]
    L.ppcg_solve.argtypes = [PG, P, P, P, S, P, C.POINTER(PpcgInfo), P]
    L.hydro_conservation_work_bytes.argtypes = [PT]
    L.hydro_conservation_work_bytes.restype = S
    L.hydro_conservation.argtypes = [PT, P, P, P, S, C.c_int32, P]
    L.hydro_restrict_complete.argtypes = [PT, P, P]
    L.hydro_state_to_fp32.argtypes = [P, P, C.c_int64, P]
    L.hydro_state_from_fp32.argtypes = [P, P, C.c_int64, P]
    L.amr_get_status.argtypes = [PP, P, P]
    L.amr_status_string.argtypes = [C.c_int]
    L.amr_status_string.restype = C.c_char_p
    for name in EXPORTS:
        if name not in ("hydro_flux_reg_bytes", "amr_status_string", "mlp_packed_bytes", "mlp_scratch_bytes",
                        "ppcg_workspace_bytes", "amr_refine_work_bytes", "hydro_conservation_work_bytes"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


class AmrError(RuntimeError):
    def __init__(self, call, status):
        self.status = status
        msg = lib().amr_status_string(status).decode()
        super().__init__("%s failed: %s (%d)" % (call, msg, status))


def check(call, status):
    if status != OK:
        raise AmrError(call, status)
