"""Seeded synthetic inputs shared by the oracle tests, the CUDA parity tests and bench.py.

Holds none of the method's arithmetic: only random parameters of the analytic initial
conditions (Fourier modes on a constant state, four-quadrant Riemann states) and random
refinement flags.
"""
import numpy as np

# paper workloads (Sec. 4): parameters of the analytic initial conditions
VORTEX = [5.0, 5.0, 5.0, 1.0, 1.0, 1.0, 1.0]          # eps, centre, background rho, u, v, p
EXPLOSION = [0.5, 1.0, 1.0, 0.125, 0.1]                # R, rho_in, p_in, rho_out, p_out


def base_state(dim, pde):
    if pde == "euler":
        return [1.0] + [0.3, -0.2, 0.1][:dim] + [1.0]
    if pde == "mhd":
        return [1.0, 0.3, -0.2, 0.0, 1.0, 0.4, -0.3, 0.0, 0.0]
    return [1.0]


def fourier_params(seed, dim, pde, nmodes=4, amp=0.05):
    """base primitive state + nmodes small sine modes with random wave numbers and phases"""
    rng = np.random.default_rng(seed)
    base = base_state(dim, pde)
    V = len(base)
    out = list(base) + [float(nmodes)]
    for _ in range(nmodes):
        var = int(rng.integers(0, V))
        k = [int(rng.integers(0, 3)) for _ in range(3)]
        if dim == 2:
            k[2] = 0
        if not any(k[:dim]):
            k[0] = 1
        out += [float(var), float(k[0]), float(k[1]), float(k[2]), float(amp * rng.uniform(0.5, 1.0)),
                float(rng.uniform(0, 2 * np.pi))]
    return out


def rp4_params(seed):
    """four-quadrant Riemann data: rho, p ~ U[0.1, 1.5], u, v ~ U[-1, 1] per quadrant"""
    rng = np.random.default_rng(seed)
    out = [0.0, 0.0]
    for _ in range(4):
        out += [rng.uniform(0.1, 1.5), rng.uniform(-1, 1), rng.uniform(-1, 1), rng.uniform(0.1, 1.5)]
    return out


def random_flags(rng, meta, p_refine=0.1, p_coarsen=0.5):
    """random flags in canonical order: +1 on a fraction of active cells, -1 on a fraction of
    virtual mothers"""
    n = len(meta)
    f = np.zeros(n, dtype=np.int8)
    f[(meta[:, 1] == 0) & (rng.random(n) < p_refine)] = 1
    f[(meta[:, 1] == -1) & (rng.random(n) < p_coarsen)] = -1
    return f
