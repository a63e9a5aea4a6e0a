"""Helpers of the adjoint tests: vector-Jacobian products and gradients of the FP64 oracle
(torch autograd through the oracle's steps) at the same states as the GPU library."""
import numpy as np
import torch

from oracle import fd as ofd
from oracle.step import Oracle


def lattice_w(o):
    return np.array([o.lat.w[i].item() for i in range(o.lat.Q)])


def _sizes(wl):
    th = bool(wl.cfg.get("thermal"))
    return wl.N, wl.Q, wl.cfg["dim"], (len(wl.cfg["species"]) if th else 0), th


def state_from_buffer(o, wl, buf, dtype):
    """Oracle state dict from a device buffer in the lbm_save_state layout (fields of the storage
    type: populations in the shifted form q = g / w - P_ref, then u, and T, Y when thermal).
    P_th, dP_lag and M are those of the open-domain oracle (constants)."""
    N, Q, D, K, th = _sizes(wl)
    n = (Q + D + (1 + K if th else 0)) * N
    a = buf[: n * dtype.itemsize].view(dtype).double().cpu()
    w = torch.as_tensor(lattice_w(o))[:, None]
    P_ref = wl.cfg.get("P_ref", 0.0)
    st = o.init_state(T=wl.T, Y=wl.Y, u=wl.u, P_h=wl.P_h, g_pert=wl.g_pert)
    fl = o.grid.fluid
    # fluid cells from the buffer; solid cells keep the initial values (no step reads them)
    st["g"] = torch.where(fl[None, :], w * (a[: Q * N].reshape(Q, N) + P_ref), st["g"])
    st["u"] = torch.where(fl[None, :], a[Q * N:(Q + D) * N].reshape(D, N), st["u"])
    if th:
        st["T"] = torch.where(fl, a[(Q + D) * N:(Q + D + 1) * N], st["T"])
        st["Y"] = torch.where(fl[None, :], a[(Q + D + 1) * N:n].reshape(K, N), st["Y"])
    return st


def seeded_adjoint(wl, seed):
    """Random adjoint of a state, zero on solid cells (oracle form: adjoint of g)."""
    rng = np.random.default_rng(seed)
    N, Q, D, K, th = _sizes(wl)
    fl = (np.asarray(wl.mask).reshape(-1) == 0).astype(np.float64)
    lam = {"g": rng.standard_normal((Q, N)) * fl, "u": rng.standard_normal((D, N)) * fl}
    if th:
        lam["T"] = rng.standard_normal(N) * fl
        lam["Y"] = rng.standard_normal((K, N)) * fl
    return lam


def pack_adjoint(o, lam):
    """The adjoint in the lbm_save_state layout: the populations are stored as q = g / w - P_ref,
    so the adjoint of q_i is w_i times the adjoint of g_i."""
    w = lattice_w(o)
    parts = [(lam["g"] * w[:, None]).ravel(), lam["u"].ravel()]
    if "T" in lam:
        parts += [lam["T"].ravel(), lam["Y"].ravel()]
    return np.concatenate(parts)


def unpack_adjoint(o, wl, a):
    N, Q, D, K, th = _sizes(wl)
    w = lattice_w(o)
    out = {"g": a[: Q * N].reshape(Q, N) / w[:, None], "u": a[Q * N:(Q + D) * N].reshape(D, N)}
    if th:
        out["T"] = a[(Q + D) * N:(Q + D + 1) * N]
        out["Y"] = a[(Q + D + 1) * N:(Q + D + 1 + K) * N].reshape(K, N)
    return out


def _inlet_leaf(o):
    inlet = o.inlet_face.detach().clone().requires_grad_()
    o.inlet_face = inlet
    o.uin_r = inlet[:, o.grid.face_index()]
    return inlet


def oracle_vjp(o, st, lam):
    """Gradient of sum(lam . step(state)) with respect to the state and the inlet face."""
    leaf = {k: st[k].detach().clone().requires_grad_() for k in ("g", "u", "T", "Y") if k in lam}
    inlet = _inlet_leaf(o)
    s = dict(st)
    s.update(leaf)
    new = o.step(s)
    L = sum((torch.as_tensor(lam[k]) * new[k]).sum() for k in lam)
    L.backward()
    out = {k: leaf[k].grad.numpy() for k in leaf}
    out["inlet"] = inlet.grad.numpy()
    return out


def oracle_fuel_gradient(wl, n_steps, fuel, inlet_u=None, T0=None):
    """J = sum over fluid cells of -omega_fuel after n_steps from (inlet_u, T0), and its
    gradient with respect to both, by autograd through the oracle."""
    o = Oracle(wl.cfg, wl.mask, wl.inlet_u if inlet_u is None else inlet_u)
    inlet = _inlet_leaf(o)
    T0 = torch.as_tensor(wl.T if T0 is None else T0, dtype=torch.float64).reshape(-1).clone().requires_grad_()
    st = o.init_state(T=T0, Y=wl.Y, u=wl.u, P_h=wl.P_h, g_pert=wl.g_pert)
    for _ in range(n_steps):
        st = o.step(st)
    J = ofd.fuel_consumption(o.p, st["T"], st["Y"], st["P_th"], o.grid.fluid, fuel)
    J.backward()
    return J.item(), inlet.grad.numpy(), T0.grad.numpy()
