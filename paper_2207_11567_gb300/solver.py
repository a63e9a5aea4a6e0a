"""Python face of the C ABI: a ``Solver`` that owns one library context.

PyTorch provides device memory (the caching allocator, through the ABI's allocator hooks) and
the CUDA stream; every step of the method runs in the library's CUDA kernels.
"""
import ctypes as C

import numpy as np
import torch

from . import _lib as L


def _check(ctx, status):
    if status != L.LBM_OK:
        msg = L.lib.lbm_last_error(ctx).decode() if ctx else ""
        raise L.HLBMError(status, msg)


class _TorchAllocator:
    """Device allocations through torch's caching allocator on one stream."""

    def __init__(self, device, stream):
        self.device, self.stream = device, stream
        self.alloc = L.ALLOC_FN(self._alloc)
        self.free = L.FREE_FN(self._free)

    def _alloc(self, nbytes, _user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream)
        except Exception:  # out of memory: the library reports LBM_ERR_ALLOC
            return None

    def _free(self, ptr, _user):
        torch.cuda.caching_allocator_delete(ptr)


def _as_c_double(arr):
    """Host float64 contiguous array and its pointer (the array must be kept alive)."""
    a = np.ascontiguousarray(np.asarray(arr, dtype=np.float64))
    return a, a.ctypes.data_as(C.c_void_p)


class Solver:
    """One simulation context (``include/hlbm.h``)."""

    def __init__(self, cfg, mask, inlet_u=None, device=None, stream=None, torch_alloc=True):
        if not torch.cuda.is_available():
            raise RuntimeError("the hybrid LB/FD library needs a CUDA device")
        self.cfg = cfg
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
            self._c = L.config_from_dict(cfg, C.c_void_p(self.stream.cuda_stream))
            self._alloc = None
            if torch_alloc:
                self._alloc = _TorchAllocator(self.device, self.stream)
                self._c.alloc, self._c.free = self._alloc.alloc, self._alloc.free
            self.ctx = C.c_void_p()
            st = L.lib.lbm_init(C.byref(self._c), C.byref(self.ctx))
            if st != L.LBM_OK:
                msg = L.lib.lbm_last_error(self.ctx).decode() if self.ctx else ""
                L.lib.lbm_destroy(self.ctx)
                self.ctx = None
                raise L.HLBMError(st, msg)
        self.dim = cfg["dim"]
        self.Q = 3 ** self.dim
        self.K = len(cfg.get("species", [])) if cfg.get("thermal") else 0
        nz = cfg.get("nz", 1) if self.dim == 3 else 1
        self.N = cfg["nx"] * cfg["ny"] * nz
        if cfg.get("variable_cp"):
            self.set_thermo([sp["cp_poly"] for sp in cfg["species"]], cfg.get("T0_thermo", 298.15))
        if cfg.get("mixture_averaged"):
            self.set_transport(cfg["Le_pair"])
        self.set_geometry(mask, inlet_u)

    def __del__(self):
        self.close()

    def close(self):
        if getattr(self, "ctx", None):
            L.lib.lbm_destroy(self.ctx)
            self.ctx = None

    # ---------------------------------------------------------------------------- set-up
    def set_geometry(self, mask, inlet_u=None):
        m = np.ascontiguousarray(np.asarray(mask, dtype=np.uint8).reshape(-1))
        if m.size != self.N:
            raise ValueError("mask size")
        keep = None
        ptr = None
        if inlet_u is not None:
            keep, ptr = _as_c_double(inlet_u)
        with torch.cuda.device(self.device):
            _check(self.ctx, L.lib.lbm_set_geometry(self.ctx, m.ctypes.data_as(C.c_void_p), ptr, 0))
        del keep

    def set_thermo(self, cp_poly, T0=298.15):
        """Variable heat capacities (lbm_set_thermo): cp_poly [n_species][5] coefficients of
        c_p,k(T) = sum_m a_m T^m in J/(kg K), formation enthalpies at T0; None for constant c_p."""
        if cp_poly is None:
            _check(self.ctx, L.lib.lbm_set_thermo(self.ctx, None, float(T0)))
            return
        a = np.zeros((len(self.cfg["species"]), 5))
        for k, row in enumerate(cp_poly):
            a[k, : len(row)] = row
        keep, ptr = _as_c_double(a)
        _check(self.ctx, L.lib.lbm_set_thermo(self.ctx, ptr, float(T0)))
        del keep

    def set_transport(self, Le_pair):
        """Mixture-averaged species diffusion with pair Lewis numbers Le_pair [n_species][n_species]
        (lbm_set_transport); None for the constant Lewis numbers of the configuration."""
        if Le_pair is None:
            _check(self.ctx, L.lib.lbm_set_transport(self.ctx, None))
            return
        K = len(self.cfg["species"])
        keep, ptr = _as_c_double(np.asarray(Le_pair, dtype=np.float64).reshape(K, K))
        _check(self.ctx, L.lib.lbm_set_transport(self.ctx, ptr))
        del keep

    def set_inlet(self, inlet_u):
        """Replace the inlet-face velocities [dim][ny nz] (lattice units) between steps
        (lbm_set_inlet); fields and captured graphs stay."""
        keep, ptr = _as_c_double(inlet_u)
        if keep.size != self.N // self.cfg["nx"] * self.dim:
            raise ValueError("inlet size")
        with torch.cuda.device(self.device):
            _check(self.ctx, L.lib.lbm_set_inlet(self.ctx, ptr, 0))
        del keep

    def set_wall_fractions(self, q):
        """Interpolated bounce-back: q [Q][N] wall fraction per bounce-back link (0.5 half-way),
        or None to clear (lbm_set_wall_fractions). Call after set_geometry."""
        keep, ptr = (None, None) if q is None else _as_c_double(q)
        with torch.cuda.device(self.device):
            _check(self.ctx, L.lib.lbm_set_wall_fractions(self.ctx, ptr))
        del keep

    def set_wall_links(self, cell, direction, q):
        """Interpolated bounce-back from a list of links (lbm_set_wall_links): cell index, pull
        direction and wall fraction of each link."""
        c = np.ascontiguousarray(np.asarray(cell, dtype=np.int32))
        d = np.ascontiguousarray(np.asarray(direction, dtype=np.int32))
        v = np.ascontiguousarray(np.asarray(q, dtype=np.float64))
        if not (c.size == d.size == v.size):
            raise ValueError("cell, direction and q must have the same length")
        with torch.cuda.device(self.device):
            _check(self.ctx, L.lib.lbm_set_wall_links(self.ctx, int(c.size), c.ctypes.data_as(C.c_void_p),
                                                      d.ctypes.data_as(C.c_void_p), v.ctypes.data_as(C.c_void_p)))

    def set_fields(self, T=None, Y=None, u=None, P_h=None, g_pert=None):
        keep = []

        def p(a):
            if a is None:
                return None
            arr, ptr = _as_c_double(a)
            keep.append(arr)
            return ptr

        if u is None:
            u = np.zeros((self.dim, self.N))
        if P_h is None:
            P_h = np.zeros(self.N)
        with torch.cuda.device(self.device):
            _check(self.ctx, L.lib.lbm_set_fields(self.ctx, p(T), p(Y), p(u), p(P_h), p(g_pert), 0))

    # ------------------------------------------------------------------------------ run
    def step(self, n=1):
        with torch.cuda.device(self.device):
            _check(self.ctx, L.lib.lbm_step(self.ctx, int(n)))

    def synchronize(self):
        self.stream.synchronize()

    def _after_torch(self):
        """Order the context's stream after work already queued on torch's current stream."""
        self.stream.wait_stream(torch.cuda.current_stream(self.device))

    def _before_torch(self):
        """Order torch's current stream after the work queued on the context's stream."""
        torch.cuda.current_stream(self.device).wait_stream(self.stream)

    # --------------------------------------------------------------------------- output
    def fields(self, bits=L.F_T | L.F_Y | L.F_U | L.F_PH | L.F_RHO | L.F_LAM | L.F_G, device=False, out=None):
        """Selected fields as float64 (numpy on the host, or a torch tensor on the device). out: an
        optional host float64 array of lbm_fields_size(bits) values to fill (e.g. pinned memory)."""
        if not self.cfg.get("thermal"):
            bits &= ~(L.F_T | L.F_Y | L.F_RHO | L.F_LAM)
        n = L.lib.lbm_fields_size(self.ctx, bits)
        with torch.cuda.device(self.device):
            if out is not None:
                buf = np.asarray(out).reshape(-1)
                if buf.dtype != np.float64 or buf.size < n or not buf.flags.c_contiguous:
                    raise ValueError("out must be a contiguous float64 array of at least %d values" % n)
                buf = buf[:n]
                _check(self.ctx, L.lib.lbm_get_fields(self.ctx, bits, buf.ctypes.data_as(C.c_void_p), 0))
            elif device:
                out = torch.empty(n, dtype=torch.float64, device=self.device)
                self._after_torch()
                _check(self.ctx, L.lib.lbm_get_fields(self.ctx, bits, C.c_void_p(out.data_ptr()), 1))
                self._before_torch()
                buf = out
            else:
                buf = np.empty(n, dtype=np.float64)
                _check(self.ctx, L.lib.lbm_get_fields(self.ctx, bits, buf.ctypes.data_as(C.c_void_p), 0))
        res, off, N = {}, 0, self.N
        for bit, name, count in ((L.F_T, "T", 1), (L.F_Y, "Y", self.K), (L.F_U, "u", self.dim),
                                 (L.F_PH, "P_h", 1), (L.F_RHO, "rho", 1), (L.F_LAM, "lam", 1),
                                 (L.F_G, "g", self.Q)):
            if bits & bit:
                v = buf[off: off + count * N]
                res[name] = v.reshape(count, N) if count != 1 or name in ("Y",) else v
                off += count * N
        return res

    def scalars(self):
        out = (C.c_double * 4)()
        with torch.cuda.device(self.device):
            _check(self.ctx, L.lib.lbm_get_scalars(self.ctx, out))
        return {"P_th": out[0], "dP": out[1], "M": out[2], "steps": int(out[3])}

    def links(self):
        out = np.empty(self.N, dtype=np.uint32)
        with torch.cuda.device(self.device):
            _check(self.ctx, L.lib.lbm_get_links(self.ctx, out.ctypes.data_as(C.c_void_p), 0))
        return out

    def stencil_words(self):
        out = np.empty(self.N, dtype=np.uint32)
        with torch.cuda.device(self.device):
            _check(self.ctx, L.lib.lbm_get_stencil_words(self.ctx, out.ctypes.data_as(C.c_void_p), 0))
        return out

    # ----------------------------------------------------------------------- diagnostics
    def stats_control(self, op, interval=1):
        """0 reset, 1 sample every `interval` steps, 2 stop (lbm_stats_control)."""
        _check(self.ctx, L.lib.lbm_stats_control(self.ctx, int(op), int(interval)))

    def stats(self):
        """(mean, rms, n): arrays [nf][N] for u components, P_h (and T), and the sample count."""
        nf = self.dim + 1 + (1 if self.cfg.get("thermal") else 0)
        buf = np.empty(2 * nf * self.N, dtype=np.float64)
        n = C.c_longlong()
        with torch.cuda.device(self.device):
            _check(self.ctx, L.lib.lbm_get_stats(self.ctx, buf.ctypes.data_as(C.c_void_p), 0, C.byref(n)))
        return buf[: nf * self.N].reshape(nf, self.N), buf[nf * self.N:].reshape(nf, self.N), n.value

    def flame_length(self, level, T_u, T_b):
        """Length (cells) of the c = level iso-line of c = (T - T_u) / (T_b - T_u) (2-D)."""
        out = C.c_double()
        with torch.cuda.device(self.device):
            _check(self.ctx, L.lib.lbm_flame_length(self.ctx, float(level), float(T_u), float(T_b), C.byref(out)))
        return out.value

    def set_probes(self, cells, capacity=65536, interval=1):
        """Record u, P_h (and T) at the given fluid cells after every `interval`-th step into a
        ring of `capacity` samples (lbm_set_probes); an empty list stops recording."""
        c = np.ascontiguousarray(np.asarray(cells, dtype=np.int32).reshape(-1))
        with torch.cuda.device(self.device):
            _check(self.ctx, L.lib.lbm_set_probes(self.ctx, int(c.size), c.ctypes.data_as(C.c_void_p),
                                                  int(capacity), int(interval)))
        self._probe_count, self._probe_interval = int(c.size), int(interval)

    def probes(self):
        """Recorded samples, oldest first: array [n_samples][n_probes][nf], fields u_x, u_y[, u_z],
        P_h[, T]."""
        n = C.c_longlong()
        with torch.cuda.device(self.device):
            _check(self.ctx, L.lib.lbm_get_probes(self.ctx, None, 0, C.byref(n)))
            nf = self.dim + 1 + (1 if self.cfg.get("thermal") else 0)
            out = np.empty(n.value * nf * self._probe_count, dtype=np.float64)
            if out.size:
                self._after_torch()
                _check(self.ctx, L.lib.lbm_get_probes(self.ctx, out.ctypes.data_as(C.c_void_p), 0, C.byref(n)))
        return out.reshape(n.value, -1, nf) if out.size else out.reshape(0, 0, nf)

    def welch_psd(self, x, dt, seg_len, stride=1):
        """Welch power spectral density of a device tensor x (float64, 1-D; every `stride`-th
        element), lbm_welch_psd; returns (frequencies in Hz, psd)."""
        if x.dtype != torch.float64 or not x.is_cuda:
            raise ValueError("x must be a float64 CUDA tensor")
        n = (x.numel() + stride - 1) // stride
        psd = np.empty(seg_len // 2 + 1)
        with torch.cuda.device(self.device):
            self._after_torch()
            _check(self.ctx, L.lib.lbm_welch_psd(self.ctx, C.c_void_p(x.data_ptr()), n, stride, float(dt),
                                                 int(seg_len), psd.ctypes.data_as(C.c_void_p)))
        return np.arange(psd.size) / (seg_len * dt), psd

    def probe_spectrum(self, probe, field, seg_len):
        """Welch spectrum of one probe's field over the recorded samples (lbm_probe_spectrum);
        returns (frequencies in Hz, psd)."""
        psd = np.empty(seg_len // 2 + 1)
        with torch.cuda.device(self.device):
            _check(self.ctx, L.lib.lbm_probe_spectrum(self.ctx, int(probe), int(field), int(seg_len),
                                                      psd.ctypes.data_as(C.c_void_p)))
        return np.arange(psd.size) / (seg_len * self.cfg["dt"] * self._probe_interval), psd

    def flame_properties(self, fuel=0, profile=False):
        """Planar flame along x (lbm_flame_properties): dict with S_c (m/s), delta_L (m), x_f (m),
        T_min, T_max, T_b and Y_b [K]; with profile=True also the column means T, w_F (fuel
        consumption rate -omega_F, kg/(m^3 s)) and Y [K][nx]."""
        K = len(self.cfg["species"])
        nx = self.cfg["nx"]
        props = np.zeros(6 + K)
        prof = np.zeros((2 + K, nx)) if profile else None
        with torch.cuda.device(self.device):
            self._after_torch()
            _check(self.ctx, L.lib.lbm_flame_properties(
                self.ctx, int(fuel), props.ctypes.data_as(C.c_void_p),
                prof.ctypes.data_as(C.c_void_p) if profile else None))
        out = {"S_c": props[0], "delta_L": props[1], "x_f": props[2], "T_min": props[3], "T_max": props[4],
               "T_b": props[5], "Y_b": props[6:].copy()}
        if profile:
            out.update({"T": prof[0].copy(), "w_F": prof[1].copy(), "Y": prof[2:].copy()})
        return out

    # ---------------------------------------------------------------------- checkpoints
    def state_bytes(self):
        return int(L.lib.lbm_state_bytes(self.ctx))

    def save_state(self, buf=None):
        if buf is None:
            buf = torch.empty(self.state_bytes(), dtype=torch.uint8, device=self.device)
        with torch.cuda.device(self.device):
            self._after_torch()
            _check(self.ctx, L.lib.lbm_save_state(self.ctx, C.c_void_p(buf.data_ptr())))
            self._before_torch()
        return buf

    def load_state(self, buf):
        with torch.cuda.device(self.device):
            self._after_torch()
            _check(self.ctx, L.lib.lbm_load_state(self.ctx, C.c_void_p(buf.data_ptr())))
            self._before_torch()

    # --------------------------------------------------------------------------- adjoint
    def adjoint_step(self, state_n, adj, grad_inlet):
        """Reverse of one step from the saved state ``state_n`` (lbm_adjoint_step): ``adj``
        (device tensor in the lbm_save_state layout and storage type) holds the adjoint of the
        state after the step and is overwritten with the adjoint of ``state_n``; the adjoint of
        the inlet-face velocity is added into ``grad_inlet`` ([dim][ny], storage type)."""
        with torch.cuda.device(self.device):
            self._after_torch()
            _check(self.ctx, L.lib.lbm_adjoint_step(self.ctx, C.c_void_p(state_n.data_ptr()),
                                                    C.c_void_p(adj.data_ptr()), C.c_void_p(grad_inlet.data_ptr())))
            self._before_torch()

    def adjoint_segment(self, checkpoint, n_steps, adj, grad_inlet):
        """Reverse sweep over n_steps steps from the saved state ``checkpoint``
        (lbm_adjoint_segment): ``adj`` holds the adjoint of the state n_steps later and is
        overwritten with that of ``checkpoint``; the inlet adjoint is added into ``grad_inlet``."""
        with torch.cuda.device(self.device):
            self._after_torch()
            _check(self.ctx, L.lib.lbm_adjoint_segment(self.ctx, C.c_void_p(checkpoint.data_ptr()), int(n_steps),
                                                       C.c_void_p(adj.data_ptr()), C.c_void_p(grad_inlet.data_ptr())))
            self._before_torch()

    def adjoint_sweep(self, checkpoints, seg_len, n_steps, adj, grad_inlet):
        """Reverse sweep over a whole run from its checkpoints (lbm_adjoint_sweep): checkpoints[s]
        is the saved state s * seg_len; ``adj`` holds the adjoint of state n_steps and is
        overwritten with that of state 0; the inlet adjoint is added into ``grad_inlet``. The
        recompute of each segment overlaps the reverse of the one after it."""
        ptrs = (C.c_void_p * len(checkpoints))(*[c.data_ptr() for c in checkpoints])
        with torch.cuda.device(self.device):
            self._after_torch()
            _check(self.ctx, L.lib.lbm_adjoint_sweep(self.ctx, ptrs, len(checkpoints), int(seg_len), int(n_steps),
                                                     C.c_void_p(adj.data_ptr()), C.c_void_p(grad_inlet.data_ptr())))
            self._before_torch()

    def initial_T_adjoint(self, state0, adj0, grad_T0):
        """dJ/dT0 into ``grad_T0`` ([N], storage type) from the adjoint ``adj0`` of the state
        ``state0`` that set_fields produced (lbm_initial_T_adjoint)."""
        with torch.cuda.device(self.device):
            self._after_torch()
            _check(self.ctx, L.lib.lbm_initial_T_adjoint(self.ctx, C.c_void_p(state0.data_ptr()),
                                                         C.c_void_p(adj0.data_ptr()), C.c_void_p(grad_T0.data_ptr())))
            self._before_torch()

    def fuel_objective(self, fuel, adj_out):
        """J = sum over fluid cells of -omega_fuel for the current state; its gradient with
        respect to the state is written to ``adj_out`` (lbm_save_state layout). Returns J."""
        J = C.c_double()
        with torch.cuda.device(self.device):
            self._after_torch()
            _check(self.ctx, L.lib.lbm_fuel_objective(self.ctx, int(fuel), C.byref(J), C.c_void_p(adj_out.data_ptr())))
            self._before_torch()
        return J.value

    # ------------------------------------------------------------------------- profiling
    def profile(self, enable=True):
        _check(self.ctx, L.lib.lbm_profile(self.ctx, int(enable)))

    def kernel_times(self):
        ms = (C.c_double * L.KERNEL_KINDS)()
        n = (C.c_longlong * L.KERNEL_KINDS)()
        _check(self.ctx, L.lib.lbm_kernel_times(self.ctx, ms, n))
        return {L.KERNEL_NAMES[k]: (ms[k], n[k]) for k in range(L.KERNEL_KINDS)}

    def kernel_bytes(self):
        b = (C.c_double * L.KERNEL_KINDS)()
        _check(self.ctx, L.lib.lbm_kernel_bytes(self.ctx, b))
        return {L.KERNEL_NAMES[k]: b[k] for k in range(L.KERNEL_KINDS)}

    def use_graphs(self, enable=True):
        _check(self.ctx, L.lib.lbm_use_graphs(self.ctx, int(enable)))


def from_workload(wl, **kw):
    """Solver initialised with a ``workloads.Workload``'s geometry and fields."""
    s = Solver(wl.cfg, wl.mask, wl.inlet_u, **kw)
    if getattr(wl, "qwall", None) is not None:
        s.set_wall_fractions(wl.qwall)
    elif wl.info.get("wall_links") is not None:
        s.set_wall_links(*wl.info["wall_links"])
    s.set_fields(T=wl.T, Y=wl.Y, u=wl.u, P_h=wl.P_h, g_pert=wl.g_pert)
    return s
