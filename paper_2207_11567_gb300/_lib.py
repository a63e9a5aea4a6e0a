"""ctypes declarations of the C ABI in include/hlbm.h (argument marshalling only).

The shared library is built in-tree by ``build.py``; importing this module loads it and fails
loudly when it is missing. There is no CPU fallback.
"""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhlbm.so")

MAX_SPECIES = 8
MAX_REACTIONS = 4
KERNEL_KINDS = 4
KERNEL_NAMES = ("fd_update", "flame_sensor", "pth_update", "lb_stream_collide")

LBM_OK, LBM_ERR_ARG, LBM_ERR_ALLOC, LBM_ERR_CUDA, LBM_ERR_STATE, LBM_ERR_NONFINITE, LBM_ERR_UNSUPPORTED, LBM_ERR_TIMEOUT = range(8)
STATUS_NAMES = {0: "OK", 1: "ERR_ARG", 2: "ERR_ALLOC", 3: "ERR_CUDA", 4: "ERR_STATE", 5: "ERR_NONFINITE",
                6: "ERR_UNSUPPORTED", 7: "ERR_TIMEOUT"}
BC = {"periodic": 0, "wall": 1, "inlet": 2, "outlet": 3}
STORAGE = {"f64": 0, "f32": 1, "f16": 2}
COLLISION = {"bgk": 0, "cumulant": 1}
F_T, F_Y, F_U, F_PH, F_RHO, F_LAM, F_G = 1, 2, 4, 8, 16, 32, 64

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class Species(C.Structure):
    _fields_ = [("W", C.c_double), ("Le", C.c_double), ("hf", C.c_double)]


class Reaction(C.Structure):
    _fields_ = [("A", C.c_double), ("beta", C.c_double), ("E", C.c_double),
                ("nu", C.c_double * MAX_SPECIES), ("order", C.c_double * MAX_SPECIES)]


class Config(C.Structure):
    _fields_ = [
        ("dim", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("storage", C.c_int), ("collision", C.c_int),
        ("bc_lo", C.c_int * 3), ("bc_hi", C.c_int * 3),
        ("thermal", C.c_int),
        ("dx", C.c_double), ("dt", C.c_double), ("nu_ref", C.c_double),
        ("T_ref", C.c_double), ("mu_exp", C.c_double), ("Pr", C.c_double), ("cp", C.c_double),
        ("rho_ref", C.c_double), ("P_th0", C.c_double), ("P_ref", C.c_double),
        ("smag_cs", C.c_double), ("omega_bulk", C.c_double), ("omega_hi", C.c_double * 4),
        ("thicken_F", C.c_double), ("flame_sensor", C.c_int), ("sensor_species", C.c_int),
        ("sensor_oxidizer", C.c_int), ("sensor_beta", C.c_double), ("sensor_wref", C.c_double),
        ("sensor_Ta", C.c_double),
        ("closed_domain", C.c_int), ("n_species", C.c_int), ("n_reactions", C.c_int),
        ("sp", Species * MAX_SPECIES), ("rx", Reaction * MAX_REACTIONS),
        ("T_in", C.c_double), ("Y_in", C.c_double * MAX_SPECIES),
        ("stream", C.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_user", C.c_void_p),
    ]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_2207_11567_gb300.build.build()")
    lib = C.CDLL(LIB_PATH)
    P = C.c_void_p
    sig = {
        "lbm_init": (C.c_int, [C.POINTER(Config), C.POINTER(P)]),
        "lbm_destroy": (None, [P]),
        "lbm_last_error": (C.c_char_p, [P]),
        "lbm_set_geometry": (C.c_int, [P, P, P, C.c_int]),
        "lbm_set_fields": (C.c_int, [P, P, P, P, P, P, C.c_int]),
        "lbm_step": (C.c_int, [P, C.c_int]),
        "lbm_fields_size": (C.c_size_t, [P, C.c_uint]),
        "lbm_get_fields": (C.c_int, [P, C.c_uint, P, C.c_int]),
        "lbm_get_scalars": (C.c_int, [P, C.POINTER(C.c_double)]),
        "lbm_get_links": (C.c_int, [P, P, C.c_int]),
        "lbm_get_stencil_words": (C.c_int, [P, P, C.c_int]),
        "lbm_state_bytes": (C.c_size_t, [P]),
        "lbm_save_state": (C.c_int, [P, P]),
        "lbm_load_state": (C.c_int, [P, P]),
        "lbm_profile": (C.c_int, [P, C.c_int]),
        "lbm_kernel_times": (C.c_int, [P, C.POINTER(C.c_double), C.POINTER(C.c_longlong)]),
        "lbm_kernel_bytes": (C.c_int, [P, C.POINTER(C.c_double)]),
        "lbm_use_graphs": (C.c_int, [P, C.c_int]),
        "lbm_adjoint_step": (C.c_int, [P, P, P, P]),
        "lbm_fuel_objective": (C.c_int, [P, C.c_int, C.POINTER(C.c_double), P]),
        "lbm_initial_T_adjoint": (C.c_int, [P, P, P, P]),
        "lbm_adjoint_segment": (C.c_int, [P, P, C.c_int, P, P]),
        "lbm_set_wall_fractions": (C.c_int, [P, P]),
        "lbm_set_wall_links": (C.c_int, [P, C.c_longlong, P, P, P]),
        "lbm_stats_control": (C.c_int, [P, C.c_int, C.c_int]),
        "lbm_get_stats": (C.c_int, [P, P, C.c_int, C.POINTER(C.c_longlong)]),
        "lbm_flame_length": (C.c_int, [P, C.c_double, C.c_double, C.c_double, C.POINTER(C.c_double)]),
        "lbm_flame_properties": (C.c_int, [P, C.c_int, P, P]),
        "lbm_set_inlet": (C.c_int, [P, P, C.c_int]),
        "lbm_set_thermo": (C.c_int, [P, P, C.c_double]),
        "lbm_set_transport": (C.c_int, [P, P]),
        "lbm_adjoint_sweep": (C.c_int, [P, P, C.c_int, C.c_int, C.c_int, P, P]),
        "lbm_set_probes": (C.c_int, [P, C.c_int, P, C.c_longlong, C.c_int]),
        "lbm_get_probes": (C.c_int, [P, P, C.c_int, C.POINTER(C.c_longlong)]),
        "lbm_welch_psd": (C.c_int, [P, P, C.c_longlong, C.c_longlong, C.c_double, C.c_int, P]),
        "lbm_probe_spectrum": (C.c_int, [P, C.c_int, C.c_int, C.c_int, P]),
        "lbm_pth_integral_noalloc": (C.c_int, [P, P, P, C.c_int, C.c_int, C.POINTER(C.c_double), C.c_double,
                                               C.c_double, P, P, C.c_char_p, C.c_size_t]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()
EXPORTED = ("lbm_init", "lbm_destroy", "lbm_last_error", "lbm_set_geometry", "lbm_set_fields", "lbm_step",
            "lbm_fields_size", "lbm_get_fields", "lbm_get_scalars", "lbm_get_links", "lbm_get_stencil_words",
            "lbm_state_bytes",
            "lbm_save_state", "lbm_load_state", "lbm_profile", "lbm_kernel_times", "lbm_kernel_bytes",
            "lbm_use_graphs", "lbm_pth_integral_noalloc", "lbm_adjoint_step", "lbm_fuel_objective",
            "lbm_initial_T_adjoint", "lbm_adjoint_segment", "lbm_set_wall_fractions",
            "lbm_set_wall_links", "lbm_stats_control", "lbm_get_stats", "lbm_flame_length",
            "lbm_flame_properties", "lbm_set_inlet", "lbm_set_probes", "lbm_get_probes", "lbm_welch_psd",
            "lbm_probe_spectrum", "lbm_set_thermo", "lbm_adjoint_sweep", "lbm_set_transport")


class HLBMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def config_from_dict(cfg, stream=None):
    """Fill the C configuration struct from a workload dictionary (SI units)."""
    c = Config()
    c.dim, c.nx, c.ny = cfg["dim"], cfg["nx"], cfg["ny"]
    c.nz = cfg.get("nz", 1) if cfg["dim"] == 3 else 1
    c.storage = STORAGE[cfg.get("storage", "f32")]
    c.collision = COLLISION[cfg.get("collision", "cumulant")]
    for a, ax in enumerate(("x", "y", "z")[: cfg["dim"]]):
        lo, hi = cfg["bc"][ax]
        c.bc_lo[a], c.bc_hi[a] = BC[lo], BC[hi]
    c.thermal = int(bool(cfg.get("thermal", False)))
    for k in ("dx", "dt", "nu_ref"):
        setattr(c, k, float(cfg[k]))
    defaults = {"T_ref": 300.0, "mu_exp": 0.7, "Pr": 0.7, "cp": 1400.0, "rho_ref": 1.0, "P_th0": 101325.0,
                "P_ref": 0.0, "smag_cs": 0.0, "omega_bulk": 1.0, "thicken_F": 1.0, "sensor_beta": 10.0,
                "sensor_wref": 1e-5, "sensor_Ta": 8400.0, "T_in": 300.0}
    for k, v in defaults.items():
        setattr(c, k, float(cfg.get(k, v)))
    for n, v in enumerate(cfg.get("omega_hi", (1.0, 1.0, 1.0, 1.0))):
        c.omega_hi[n] = float(v)
    c.flame_sensor = int(bool(cfg.get("flame_sensor", False)))
    c.sensor_species = int(cfg.get("sensor_species", 0))
    c.sensor_oxidizer = int(cfg.get("sensor_oxidizer", 1))
    c.closed_domain = int(bool(cfg.get("closed_domain", False)))
    sp = cfg.get("species", [])
    rx = cfg.get("reactions", [])
    if len(sp) > MAX_SPECIES or len(rx) > MAX_REACTIONS:
        raise ValueError("too many species or reactions")
    c.n_species, c.n_reactions = len(sp), len(rx)
    for k, s in enumerate(sp):
        c.sp[k].W, c.sp[k].Le, c.sp[k].hf = s["W"], s["Le"], s["hf"]
    for j, r in enumerate(rx):
        c.rx[j].A, c.rx[j].beta, c.rx[j].E = r["A"], r["beta"], r["E"]
        for k, v in r["nu"].items():
            c.rx[j].nu[int(k)] = float(v)
        for k, v in r["order"].items():
            c.rx[j].order[int(k)] = float(v)
    for k, v in enumerate(cfg.get("Y_in", [])):
        c.Y_in[k] = float(v)
    c.stream = stream
    return c
