"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

Grids (node coordinates, with unwrapped periodic closure or analytic ghost
layers), prescribed mesh motions (node positions and their analytic time
derivatives), and initial primitive states for the workloads the paper uses:
isentropic vortex, uniform flow, Taylor-Green vortex, a Sod-type slab and a
jet-like inflow into a quiescent box.  No step of the numerical method lives
here; both the CUDA library and the CPU oracle consume these arrays.

Layout conventions: node arrays are ``[ndim][Nk][Nj][Ni]`` (2D: ``[2][Nj][Ni]``)
with ``N_d = n_d + 1`` on periodic axes (the last node closes the period) and
``n_d + 1 + 2 G`` on non-periodic axes (``G`` ghost node layers on each side).
States are ``[nv][nk][nj][ni]``.
"""
import math

import numpy as np

DEFAULTS = dict(
    gamma=1.4,
    prandtl=0.71,
    reynolds=0.0,
    sutherland_s=0.0,
    t_ref=1.0,
    alpha_damping=4.0,
    mp_alpha=4.0,
    mp_beta=4.0,
    mp_eps=1e-20,
    metric_scheme=0,
    ghost_nodes=10,
)

BC_ZEROGRAD = 1
BC_INFLOW = 2


def case_params(ndim, n, periodic=(1, 1, 1), bc=((1, 1), (1, 1), (1, 1)), **kw):
    c = dict(DEFAULTS)
    c.update(kw)
    c["ndim"] = int(ndim)
    n = tuple(int(v) for v in n)
    c["n"] = n + (1,) * (3 - len(n))
    c["periodic"] = tuple(int(v) for v in periodic) + (1,) * (3 - len(periodic))
    c["bc"] = tuple(tuple(int(s) for s in b) for b in bc)
    return c


# ---------------------------------------------------------------------------
# Counter-based random numbers: SplitMix64 (Steele, Lea, Flood, OOPSLA 2014)
# ---------------------------------------------------------------------------
def splitmix64(x):
    x = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = x + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def hash_uniform(seed, *keys):
    """Uniform numbers in [-1, 1) from SplitMix64 of (seed, keys...), elementwise over broadcast keys."""
    with np.errstate(over="ignore"):
        z = splitmix64(np.uint64(seed))
        for k in keys:
            z = splitmix64(z ^ np.asarray(k, dtype=np.uint64))
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 / 9007199254740992.0) - 1.0


# ---------------------------------------------------------------------------
# Grids
# ---------------------------------------------------------------------------
def _node_index(n, periodic, G):
    """Node index ranges per axis (ghost layers included)."""
    return [np.arange(-G, nd + 1 + G) if not per else np.arange(0, nd + 1) for nd, per in zip(n, periodic)]


def nodes_from_functions(n, periodic, G, fx):
    """Evaluate coordinate functions fx(I, J[, K]) -> tuple of arrays on node indices."""
    idx = _node_index(n, periodic, G)
    mesh = np.meshgrid(*idx[::-1], indexing="ij")[::-1]  # I fastest in memory
    coords = fx(*mesh)
    return np.ascontiguousarray(np.stack(coords).astype(np.float64))


def nodes_uniform(n, lengths, origin=None, periodic=None, G=10):
    nd = len(n)
    periodic = periodic or (1,) * nd
    origin = origin or (0.0,) * nd
    h = [L / m for L, m in zip(lengths, n)]
    return nodes_from_functions(n, periodic, G, lambda *I: tuple(origin[a] + I[a] * h[a] for a in range(nd)))


def nodes_wavy_2d(n=64, L=10.0, amp=0.2, wavelength=5.0):
    """x = xi + amp sin(2 pi xi / lam) sin(2 pi eta / lam), y likewise, on periodic [0, L]^2."""
    h = L / n

    def f(I, J):
        xi, eta = I * h, J * h
        s = amp * np.sin(2 * np.pi * xi / wavelength) * np.sin(2 * np.pi * eta / wavelength)
        return xi + s, eta + s

    return nodes_from_functions((n, n), (1, 1), 0, f)


def nodes_tgv_3d(n=128, amp_frac=0.1):
    """Periodic [0, 2 pi]^3; x += amp h sin(eta) sin(zeta), y, z cyclically."""
    h = 2 * np.pi / n
    A = amp_frac * h

    def f(I, J, K):
        xi, eta, zeta = I * h, J * h, K * h
        return (xi + A * np.sin(eta) * np.sin(zeta), eta + A * np.sin(zeta) * np.sin(xi),
                zeta + A * np.sin(xi) * np.sin(eta))

    return nodes_from_functions((n, n, n), (1, 1, 1), 0, f)


def nodes_sinusoidal_3d(n=20, L=4.0):
    """Sinusoidal freestream grid of the paper's 3D uniform-flow test (Sec. 8.1.1, node index = i - 1)."""
    d0 = L / n
    xmin = -L / 2

    def f(I, J, K):
        return (xmin + d0 * (I + np.sin(np.pi * J * d0) * np.sin(np.pi * K * d0)),
                xmin + d0 * (J + np.sin(np.pi * K * d0) * np.sin(np.pi * I * d0)),
                xmin + d0 * (K + np.sin(np.pi * I * d0) * np.sin(np.pi * J * d0)))

    return nodes_from_functions((n, n, n), (1, 1, 1), 0, f)


def nodes_random(n, lengths, frac=0.2, seed=7):
    """Uniform periodic grid with every node moved by up to frac * h per axis (SplitMix64)."""
    nd = len(n)
    h = [L / m for L, m in zip(lengths, n)]

    def f(*I):
        # periodic: the closing node repeats node 0's displacement
        wrapped = [np.mod(I[a], n[a]) for a in range(nd)]
        flat = wrapped[0].astype(np.uint64)
        for a in range(1, nd):
            flat = flat * np.uint64(n[a - 1] + 1) + wrapped[a].astype(np.uint64)
        out = []
        for a in range(nd):
            r = hash_uniform(seed, a, flat)
            out.append(I[a] * h[a] + frac * h[a] * r)
        return tuple(out)

    return nodes_from_functions(tuple(n), (1,) * nd, 0, f)


def nodes_skewed_2d(n, lengths, skew_deg=20.0, jitter=0.1, seed=3):
    """Affine skew (shear of x with eta) plus node jitter, periodic with a skewed period vector."""
    nx, ny = n
    Lx, Ly = lengths
    hx, hy = Lx / nx, Ly / ny
    t = math.tan(math.radians(skew_deg))

    def f(I, J):
        wi, wj = np.mod(I, nx), np.mod(J, ny)
        flat = wi.astype(np.uint64) * np.uint64(ny + 1) + wj.astype(np.uint64)
        rx = hash_uniform(seed, 0, flat)
        ry = hash_uniform(seed, 1, flat)
        x = I * hx + t * J * hy + jitter * hx * rx
        y = J * hy + jitter * hy * ry
        return x, y

    return nodes_from_functions((nx, ny), (1, 1), 0, f)


class SinusoidalMotion:
    """Prescribed node motion x_a = o_a + m_a h_a + A_a sin(2 pi w t) prod_b S_ab(m_b h_b),
    where S_ab(s) = sin(k_ab s) when k_ab != 0 and 1 otherwise (Sec. 8.2 families)."""

    def __init__(self, n, h, amp, omega, k, origin=None):
        self.nd = len(n)
        self.n = tuple(n)
        self.h = tuple(float(v) for v in h)
        self.amp = tuple(float(v) for v in amp)
        self.omega = float(omega)
        self.k = tuple(tuple(float(v) for v in row) for row in k)
        self.origin = tuple(float(v) for v in origin) if origin is not None else (0.0,) * self.nd

    def _shape(self, I):
        out = []
        for a in range(self.nd):
            s = np.ones_like(I[0], dtype=np.float64)
            for b in range(self.nd):
                if self.k[a][b] != 0.0:
                    s = s * np.sin(self.k[a][b] * (I[b] * self.h[b]))
            out.append(s)
        return out

    def nodes(self, t):
        st = math.sin(2 * math.pi * self.omega * t)

        def f(*I):
            S = self._shape(I)
            return tuple(self.origin[a] + I[a] * self.h[a] + self.amp[a] * st * S[a] for a in range(self.nd))

        return nodes_from_functions(self.n, (1,) * self.nd, 0, f)

    def velocity(self, t):
        ct = 2 * math.pi * self.omega * math.cos(2 * math.pi * self.omega * t)

        def f(*I):
            S = self._shape(I)
            return tuple(self.amp[a] * ct * S[a] for a in range(self.nd))

        return nodes_from_functions(self.n, (1,) * self.nd, 0, f)


def motion_dynamic_2d(n=256, L=10.0, T=1.0, amp=0.1):
    """x = xi + amp sin(2 pi t/T) sin(2 pi xi/L) sin(2 pi eta/L), y likewise."""
    kk = 2 * np.pi / L
    return SinusoidalMotion((n, n), (L / n, L / n), (amp, amp), 1.0 / T, ((kk, kk), (kk, kk)))


def motion_deforming_3d(n=32, L=12.0, A=1.5, nw=4, omega=1.0):
    """Sec. 8.2.1: x = xmin + dx0 [i + A sin(2 pi w t) sin(n pi j dy0/Ly) sin(n pi k dz0/Lz)], cyclic."""
    d0 = L / n
    kk = nw * np.pi / L
    k = ((0.0, kk, kk), (kk, 0.0, kk), (kk, kk, 0.0))
    return SinusoidalMotion((n, n, n), (d0, d0, d0), (A * d0,) * 3, omega, k, origin=(-L / 2,) * 3)


def stretched_axis(m, n_half=85, h0=0.02, ratio=1.02):
    """Symmetric geometric stretching about the axis node m = n_half: y = sign(s) h0 (r^|s| - 1)/(r - 1)."""
    s = np.asarray(m, dtype=np.float64) - n_half
    return np.sign(s) * h0 * (ratio ** np.abs(s) - 1.0) / (ratio - 1.0)


def nodes_jet(ni=480, nj=170, nk=170, Lx=20.0, h0=0.02, ratio=1.02, G=10):
    """Jet-like box: uniform in x on [0, Lx], symmetric geometric stretching in y and z about the
    axis, analytic continuation into G ghost node layers on every side (no periodic axis)."""
    hx = Lx / ni

    def f(I, J, K):
        return (I * hx, stretched_axis(J, nj // 2, h0, ratio), stretched_axis(K, nk // 2, h0, ratio))

    return nodes_from_functions((ni, nj, nk), (0, 0, 0), G, f)


def nodes_channel(n, lengths, amp=0.0):
    """Walls at x = 0 and x = Lx (no ghost nodes: the x axis is bounded), periodic in y (and z):
    x = xi + amp sin(pi xi / Lx) sin(2 pi eta / Ly), y = eta + amp sin(2 pi xi / Lx) sin(2 pi eta / Ly)
    (z likewise in 3D); the walls stay the planes x = 0 and x = Lx."""
    nd = len(n)
    h = [L / m for L, m in zip(lengths, n)]
    Lx = lengths[0]

    def f(*I):
        X = [I[a] * h[a] for a in range(nd)]
        wy = np.sin(2 * np.pi * X[1] / lengths[1])
        if nd == 3:
            wy = wy * np.cos(2 * np.pi * X[2] / lengths[2])
        out = [X[0] + amp * np.sin(np.pi * X[0] / Lx) * wy]
        for a in range(1, nd):
            out.append(X[a] + amp * np.sin(2 * np.pi * X[0] / Lx) * wy)
        return tuple(out)

    return nodes_from_functions(tuple(n), (0,) + (1,) * (nd - 1), 0, f)


# ---------------------------------------------------------------------------
# Cell centroids for evaluating initial conditions (input preparation only)
# ---------------------------------------------------------------------------
def centroids(nodes, n, periodic, G=10):
    """Centroids of the cells' vertices on the interior cells (periodic closures are unwrapped nodes)."""
    nd = len(n)
    X = np.asarray(nodes)
    out = []
    for c in range(nd):
        f = X[c]
        for a in range(nd):
            ax = nd - 1 - a  # array axis of index a
            off = 0 if periodic[a] else G
            f = np.take(f, np.arange(off, off + n[a] + 1), axis=ax)
        acc = np.zeros(tuple(reversed(n)))
        for corner in range(1 << nd):
            idx = []
            for a in reversed(range(nd)):
                o = (corner >> a) & 1
                idx.append(slice(o, o + n[a]))
            acc = acc + f[tuple(idx)]
        out.append(acc / (1 << nd))
    return np.stack(out)


# ---------------------------------------------------------------------------
# Initial states (primitive -> conserved with E = p/(gamma-1) + rho |u|^2 / 2)
# ---------------------------------------------------------------------------
def prim_to_cons(P, gamma):
    P = np.asarray(P, dtype=np.float64)
    nd = P.shape[0] - 2
    rho = P[0]
    u = P[1:1 + nd]
    p = P[-1]
    Q = np.empty_like(P)
    Q[0] = rho
    Q[1:1 + nd] = rho * u
    Q[-1] = p / (gamma - 1.0) + 0.5 * rho * np.sum(u * u, axis=0)
    return np.ascontiguousarray(Q)


def uniform_prim(shape, nd, gamma=1.4, mach=0.5, vel=None):
    vel = vel if vel is not None else (1.0,) + (0.0,) * (nd - 1)
    P = np.zeros((nd + 2,) + tuple(shape))
    P[0] = 1.0
    for a in range(nd):
        P[1 + a] = vel[a]
    P[-1] = 1.0 / (gamma * mach * mach)
    return P


def vortex_prim(xc, yc, gamma=1.4, mach=0.5, strength=5.0, center=(5.0, 5.0), L=10.0, t=0.0):
    """Isentropic vortex of strength eps convected by u = (1, 0) through a periodic [0, L]^2 box.
    T = p/rho; T_inf = 1/(gamma M^2); closed-form solution at time t (translation mod L)."""
    x0 = np.mod(xc - center[0] - t + L / 2, L) - L / 2
    y0 = np.mod(yc - center[1] + L / 2, L) - L / 2
    r2 = x0 * x0 + y0 * y0
    eps = strength
    Tinf = 1.0 / (gamma * mach * mach)
    du = eps / (2 * np.pi) * np.exp(0.5 * (1 - r2))
    T = Tinf - (gamma - 1) * eps * eps / (8 * gamma * np.pi * np.pi) * np.exp(1 - r2)
    rho = (T / Tinf) ** (1.0 / (gamma - 1))
    return np.stack([rho, 1.0 - du * y0, du * x0, rho * T])


def tgv_prim(xc, yc, zc, gamma=1.4, mach=0.1):
    p0 = 1.0 / (gamma * mach * mach)
    u = np.sin(xc) * np.cos(yc) * np.cos(zc)
    v = -np.cos(xc) * np.sin(yc) * np.cos(zc)
    w = np.zeros_like(u)
    p = p0 + (np.cos(2 * xc) + np.cos(2 * yc)) * (np.cos(2 * zc) + 2.0) / 16.0
    T0 = p0 / 1.0
    rho = p / T0
    return np.stack([rho, u, v, w, p])


def sod_slab_prim(s, L=1.0, x0=0.25, x1=0.75):
    """Two-sided Sod slab along coordinate s on a periodic box: (rho, p) = (1, 1) inside, (0.125, 0.1) outside.
    Returns (rho, p)."""
    s = np.mod(s, L)
    inside = (s > x0) & (s < x1)
    return np.where(inside, 1.0, 0.125), np.where(inside, 1.0, 0.1)


def jet_inflow_prim(yc, zc, gamma=1.4, p_exit=1.5, rho_exit=1.8, radius=0.5, delta=0.02):
    """Top-hat sonic inflow (p_e = 1.5, rho_e = 1.8, u_e = sqrt(gamma T_e), T_e = 2/(gamma+1)),
    smoothed with tanh over delta, into quiescent ambient rho = p = 1."""
    Te = 2.0 / (gamma + 1.0)
    ue = math.sqrt(gamma * Te)
    r = np.sqrt(yc * yc + zc * zc)
    s = 0.5 * (1.0 - np.tanh((r - radius) / delta))
    rho = 1.0 + (rho_exit - 1.0) * s
    u = ue * s
    p = 1.0 + (p_exit - 1.0) * s
    z = np.zeros_like(rho)
    return np.stack([rho, u, z, z, p])


def jet_inflow_step(base, seed, step, amp=0.01):
    """Inflow primitives of time step `step`: the base inflow [nv][nk][nj] with a random
    velocity of amplitude amp * u_base added to u, v, w, u_base the local axial inflow
    velocity (so the quiescent ambient part of the plane stays at rest).  The random numbers
    are SplitMix64 of (seed, step, cell, component) mapped to [-1, 1)."""
    base = np.asarray(base, dtype=np.float64)
    nv, nk, nj = base.shape
    cell = np.arange(nk * nj, dtype=np.uint64).reshape(nk, nj)
    out = base.copy()
    for c in (1, 2, 3):
        out[c] = base[c] + amp * base[1] * hash_uniform(seed, np.uint64(step), cell, np.uint64(c))
    return out


def jet_sponge_sigma(n, sigma_max=2.0, x_frac=0.15, lateral=10):
    """sigma = sigma_max s^2 over the last x_frac of the x cells and the outer lateral cells."""
    ni, nj, nk = n
    i = np.arange(ni)
    ix0 = int(round((1 - x_frac) * ni))
    sx = np.clip((i - ix0 + 1) / max(ni - ix0, 1), 0, 1)

    def lat(m, nm):
        d = np.minimum(m, nm - 1 - m)
        return np.clip((lateral - d) / lateral, 0, 1)

    sy = lat(np.arange(nj), nj)
    sz = lat(np.arange(nk), nk)
    S = np.maximum(np.maximum(sx[None, None, :], sy[None, :, None]), sz[:, None, None])
    return np.ascontiguousarray(sigma_max * S * S)



def jet_case(n=(480, 170, 170), Lx=20.0, h0=0.02, ratio=1.02, re_d=1e5, gamma=1.4, sutherland_s=0.3768,
             lateral=10):
    """The under-expanded jet-like workload: the stretched box of nodes_jet, quiescent ambient
    rho = p = 1 at rest, the sonic top-hat inflow of jet_inflow_prim in the x-low ghost cells,
    zero-gradient elsewhere, the sponge of jet_sponge_sigma, Sutherland viscosity with
    T_ref = T_e and mu(T_e) = rho_e u_e D / Re_D (D = 1).
    Returns (case, nodes, q, inflow, sigma, q_amb)."""
    ni, nj, nk = n
    Te = 2.0 / (gamma + 1.0)
    ue = math.sqrt(gamma * Te)
    case = case_params(3, n, periodic=(0, 0, 0), bc=((2, 1), (1, 1), (1, 1)), reynolds=re_d / (1.8 * ue),
                       sutherland_s=sutherland_s, t_ref=Te, gamma=gamma)
    nodes = nodes_jet(ni, nj, nk, Lx=Lx, h0=h0, ratio=ratio)
    xc = centroids(nodes, n, (0, 0, 0))
    inflow = np.ascontiguousarray(jet_inflow_prim(xc[1][:, :, 0], xc[2][:, :, 0], gamma))
    P = np.zeros((5, nk, nj, ni))
    P[0] = 1.0
    P[4] = 1.0
    sigma = jet_sponge_sigma(n, lateral=lateral)
    q_amb = np.array([1.0, 0.0, 0.0, 0.0, 1.0 / (gamma - 1.0)])
    return case, nodes, prim_to_cons(P, gamma), inflow, sigma, q_amb

# ---------------------------------------------------------------------------
# The serving stream: jobs of mixed kinds and sizes with Poisson arrivals
# ---------------------------------------------------------------------------
def serving_stream(n_jobs=256, seed=0, rate=1.0, edge2d=(32, 512), edge3d=(32, 128), steps=(50, 500),
                   mixed_frac=0.5):
    """Job specifications (dicts) of a serving stream.  Per job, from SplitMix64 of (seed, job, field):
    2D or 3D with equal odds; the grid edge log-uniform in edge2d / edge3d; 2D jobs are the isentropic
    vortex or a Sod slab, 3D jobs the viscous Taylor-Green vortex; an affine skew of U[0, 30] degrees
    (2D) plus 10 % node jitter; steps uniform in `steps`; FP64 or mixed precision (mixed with
    probability mixed_frac); arrivals a Poisson process of `rate` jobs per second."""
    out = []
    t = 0.0
    for j in range(n_jobs):
        u = [0.5 * (hash_uniform(seed, j, f) + 1.0) for f in range(8)]
        t += -math.log(max(1.0 - float(u[0]), 1e-300)) / rate
        nd = 2 if u[1] < 0.5 else 3
        lo, hi = edge2d if nd == 2 else edge3d
        edge = int(round(math.exp(math.log(lo) + float(u[2]) * (math.log(hi) - math.log(lo)))))
        kind = ("vortex" if u[3] < 0.5 else "sod") if nd == 2 else "tgv"
        n_steps = int(steps[0] + math.floor(float(u[4]) * (steps[1] - steps[0] + 1)))
        out.append(dict(id=j, arrival=t, ndim=nd, edge=edge, kind=kind, steps=min(n_steps, steps[1]),
                        precision="mixed" if u[5] < mixed_frac else "fp64", skew_deg=30.0 * float(u[6]),
                        seed=int(1000 + j)))
    return out


def serving_job_inputs(spec, precision=None):
    """(case, nodes, q, cfl) of one serving job (precision overrides the spec's)."""
    prec = precision or spec["precision"]
    e = spec["edge"]
    if spec["ndim"] == 2:
        n = (e, e)
        if spec["kind"] == "vortex":
            nodes = nodes_skewed_2d(n, (10.0, 10.0), skew_deg=spec["skew_deg"], jitter=0.1, seed=spec["seed"])
            xc = centroids(nodes, n, (1, 1))
            q = prim_to_cons(vortex_prim(xc[0], xc[1]), 1.4)
            cfl = 0.4
        else:
            nodes = nodes_skewed_2d(n, (1.0, 1.0), skew_deg=spec["skew_deg"], jitter=0.1, seed=spec["seed"])
            # the slab is bounded by grid lines (logical coordinate eta), oblique to x on the skewed
            # mesh; drawn on the jittered centroids instead, a row crossing the jump would hold a
            # cell-to-cell sawtooth of the two states
            eta = np.broadcast_to(((np.arange(e) + 0.5) / e)[:, None], n)
            rho, p = sod_slab_prim(eta, L=1.0)
            z = np.zeros_like(rho)
            q = prim_to_cons(np.stack([rho, z, z, p]), 1.4)
            cfl = 0.3
        case = case_params(2, n, precision=prec)
    else:
        n = (e, e, e)
        nodes = nodes_random(n, (2 * np.pi,) * 3, frac=0.1, seed=spec["seed"])
        xc = centroids(nodes, n, (1, 1, 1))
        q = prim_to_cons(tgv_prim(*xc, mach=0.1), 1.4)
        case = case_params(3, n, reynolds=1600.0, precision=prec)
        cfl = 0.2
    return case, nodes, q, cfl


def serving_job_work(spec):
    """Cell-RK-stage updates of one job."""
    return spec["edge"] ** spec["ndim"] * spec["steps"] * 3
