"""ctypes declarations of the C ABI in include/soax.h and include/soax_host.h (argument
marshalling only)."""
import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsoax.so")

STATUS_NAMES = {0: "OK", -1: "EINVAL", -2: "ESCHEMA", -3: "EALIGN", -4: "ECUDA", -5: "ETIMEOUT",
                -6: "ENOMEM", -7: "EUNSUPPORTED", -8: "EUNBOUND"}
DTYPES = {"i32": 0, "i64": 1, "u8": 2, "f32": 3, "f64": 4}


class soax_field_desc(C.Structure):
    _fields_ = [("name", C.c_char_p), ("dtype", C.c_int32), ("ncomp", C.c_int32), ("tag", C.c_char)]


class soax_flow(C.Structure):
    _fields_ = [("A", C.c_double), ("B", C.c_double), ("C", C.c_double), ("tau", C.c_double),
                ("dt", C.c_double), ("tau_scale", C.c_double), ("tau_field", C.c_int32),
                ("pos_field", C.c_int32), ("vel_field", C.c_int32), ("acc_field", C.c_int32)]


class soax_tune(C.Structure):
    _fields_ = [("parts_per_thread", C.c_int32), ("block", C.c_int32), ("vec_bits", C.c_int32),
                ("fuse_steps", C.c_int32)]


class soax_expr_op(C.Structure):
    _fields_ = [("op", C.c_int32), ("field", C.c_int32), ("comp", C.c_int32), ("pad", C.c_int32),
                ("value", C.c_double)]


EXPR_OPS = {"load": 0, "const": 1, "add": 2, "sub": 3, "mul": 4, "div": 5, "neg": 6, "abs": 7, "sqrt": 8,
            "min": 9, "max": 10, "fma": 11}

_p, _i32, _i64, _sz = C.c_void_p, C.c_int32, C.c_int64, C.c_size_t
_P = C.POINTER

# Every function include/soax.h and include/soax_host.h declare, with its argument types.
SIGNATURES = {
    "soax_version": [],
    "soax_last_error": [],
    "soax_create": [_P(soax_field_desc), _i32, _i64, _P(_p)],
    "soax_destroy": [_p],
    "soax_size": [_p, _P(_i64), _P(_i32), _P(_i32)],
    "soax_set_size": [_p, _i64],
    "soax_bind": [_p, _i32, _i32, _i32, _p],
    "soax_current": [_p, _P(_i32)],
    "soax_copy_plane": [_p, _i32, _i32, _p, _i32, _p],
    "soax_set_current": [_p, _i32],
    "soax_aos_layout": [_p, _P(_i64), _P(_i64)],
    "soax_aos_to_soa": [_p, _p, _p],
    "soax_soa_to_aos": [_p, _p, _p],
    "soax_get_element": [_p, _i64, _p, _p],
    "soax_set_element": [_p, _i64, _p, _p],
    "soax_remove_workspace_bytes": [_i64, _P(_sz)],
    "soax_remove": [_p, _p, _i64, _p, _sz, _p],
    "soax_step": [_p, _P(soax_flow), _i32, _p],
    "soax_step_fused": [_p, _P(soax_flow), _i32, _p],
    "soax_step_fused_keys": [_p, _P(soax_flow), _i32, _i32, _p, _p],
    "soax_permute_step_fused": [_p, _p, _P(soax_flow), _i32, _i32, _p, _p],
    "soax_step_aos": [_p, _p, _P(soax_flow), _i32, _p],
    "soax_cell_keys": [_p, _i32, _i32, _p, _p],
    "soax_radix_workspace_bytes": [_i64, _i32, _P(_sz)],
    "soax_radix_sort_pairs": [_p, _p, _p, _p, _i64, _i32, _p, _sz, _p],
    "soax_permute": [_p, _p, _p],
    "soax_sort_workspace_bytes": [_p, _i32, _P(_sz)],
    "soax_sort_by_keys": [_p, _i32, _p, _p, _sz, _p],
    "soax_sort_perm": [_p, _i32, _p, _p, _sz, _p],
    "soax_sort_graph_counts": [_P(C.c_int64), _P(C.c_int64)],
    "soax_sort_by_cell": [_p, _i32, _p, _sz, _p],
    "soax_sort_results": [_p, _i32, _p, _sz, _P(_p), _P(_p)],
    "soax_sort_by_cell_noalloc": [_p, _i32, _p, _p],
    "soax_fill": [_p, _i32, C.c_double, _p],
    "soax_lincomb": [_p, _i32, _i32, _i32, _p, _p, _p, C.c_double, _p],
    "soax_expr": [_p, _i32, _i32, _P(soax_expr_op), _i32, _i32, _p],
    "soax_euler": [_p, _i32, _i32, C.c_float, _i32, _p],
    "soax_euler_aos": [_p, _i64, _i64, _i64, _i64, C.c_float, _p],
    "soax_adjoint_workspace_bytes": [_p, _i32, _i32, _P(_sz)],
    "soax_step_checkpointed": [_p, _P(soax_flow), _i32, _i32, _p, _sz, _p],
    "soax_step_adjoint": [_p, _P(soax_flow), _i32, _i32, _p, _sz, _P(_p), _P(_p), _P(_p), _P(_p), _p, _p],
    "soax_minimage_loss": [_p, _i32, _P(_p), _p, _P(_p), _p, _sz, _p],
    "soax_batched_workspace_bytes": [_P(_p), _i32, _P(soax_tune), _P(_sz)],
    "soax_batched_forget": [_p],
    "soax_step_batched": [_P(_p), _P(soax_flow), _i32, _i32, _P(soax_tune), _p, _sz, _p],
    "soax_autotune": [_P(_p), _P(soax_flow), _i32, _i32, _p, _sz, _P(soax_tune), _p],
    "soax_sync": [_p],
    "soax_step_host": [_p, _P(_p), _P(soax_flow), _i32, _i32, _i32, _i32, _p, _sz, _p, _p, _p],
    "soax_step_host_finish": [_p, _p],
}
EXPORTS = list(SIGNATURES)


def declare(L):
    for name, args in SIGNATURES.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = C.c_char_p if name == "soax_last_error" else C.c_int
    return L
