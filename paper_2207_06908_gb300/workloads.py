"""Seeded synthetic inputs shared by the CUDA path, the oracle and the bench.

This module describes problems only: grid size, cell size, the material map
painted from axis-aligned blocks (the paper's "block" command, later blocks
winning), wires, source waveforms sampled in FP64 at t_{n+1/2}, probe
placements and seeded random fields.  It holds none of the update
arithmetic, coefficient rules or probe formulas of the method.

Configurations (the paper publishes no dataset; these synthetic problems
have the shapes of its grounding / lightning workloads):
  config1: 48^3 PEC box, lossy half-space, one Ez source, 3 point probes
  config2: 256^3, 10-cell CPML, air over soil, 30 m vertical thin wire fed
           at its base by a 1.2/50 us double exponential (10 kA)
  config3: 512x512x384, 12-cell CPML, two-layer soil, buried 8x8 thin-wire
           mesh with a down-conductor and the current / voltage leads of the
           paper's ground-potential-rise model
  config4: 256 grounding-rod domains of uneven size (side 48..128, 8-cell
           CPML, random soil), 2000 steps each; 512-sample impedance output
  surrogate_inputs / grounding_domain: the config-4 generator with the six
           surrogate parameters drawn as well
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

C0 = 299792458.0
PROBE_V, PROBE_I, PROBE_E, PROBE_H = 0, 1, 2, 3


@dataclasses.dataclass
class Scenario:
    name: str
    n: tuple                      # (nx, ny, nz) cells
    dx: float
    courant: float
    cpml: int                     # CPML cells (0 = PEC box)
    cell_material: np.ndarray     # (nz, ny, nx) uint8
    materials: list               # [(eps_r, sigma, mu_r)]
    wires: list = dataclasses.field(default_factory=list)     # [(p0, p1, radius)]
    sources: list = dataclasses.field(default_factory=list)   # [(node, axis, current[n] (, r_internal))]
    probes: list = dataclasses.field(default_factory=list)    # [(kind, node, axis, n_edges)]
    n_steps: int = 0
    fields: list | None = None    # optional initial [Ex,Ey,Ez,Hx,Hy,Hz] (nz,ny,nx) float32
    debye: dict = dataclasses.field(default_factory=dict)     # {material: (deps [P], tau [P] s)}
    vsources: list = dataclasses.field(default_factory=list)  # [(node, axis, voltage[n], r_internal)]
    lumped: list = dataclasses.field(default_factory=list)    # [(node, axis, resistance, capacitance)]
    wire_paths: list = dataclasses.field(default_factory=list)  # [(p0, p1, radius)] oblique, as staircases
    owires: list = dataclasses.field(default_factory=list)      # [(p0, p1, radius)] oblique wires, node units
    owire_sources: list = dataclasses.field(default_factory=list)  # [(wire, segment, emf[n](, r))] delta gaps
    owire_probes: list = dataclasses.field(default_factory=list)   # [(wire, segment)] currents, [(x, y, z)] node potentials

    @property
    def cells(self) -> int:
        return self.n[0] * self.n[1] * self.n[2]


def time_step(dx: float, courant: float) -> float:
    """The configured step: the fraction `courant` of the cubic-grid limit."""
    return courant * dx / (C0 * math.sqrt(3.0))


def sample_times(n_steps: int, dx: float, courant: float) -> np.ndarray:
    """Source sample instants t_{n+1/2}, n = 0 .. n_steps-1."""
    return (np.arange(n_steps, dtype=np.float64) + 0.5) * time_step(dx, courant)


# ---- source waveforms (inputs; FP64) ------------------------------------
def gaussian_derivative(t, tau, t0, peak=1.0):
    """-sqrt(e) ((t-t0)/tau) exp(-(t-t0)^2 / (2 tau^2)), extreme value +-peak."""
    x = (t - t0) / tau
    return -peak * math.sqrt(math.e) * x * np.exp(-0.5 * x * x)


def double_exponential_params(t_front=1.2e-6, t_half=50e-6):
    """alpha, beta, k of I(t) = I0 k (exp(-alpha t) - exp(-beta t)) with a
    front time 1.25 (t90 - t10) = t_front and the tail at half the peak at
    t_half; k normalises the peak to 1.  Solved by nested bisection."""
    def shape(alpha, beta):
        tp = math.log(beta / alpha) / (beta - alpha)
        peak = math.exp(-alpha * tp) - math.exp(-beta * tp)
        return tp, peak

    def crossing(alpha, beta, level, lo, hi):
        f = lambda t: (math.exp(-alpha * t) - math.exp(-beta * t)) - level
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if (f(lo) < 0) == (f(mid) < 0):
                lo = mid
            else:
                hi = mid
        return 0.5 * (lo + hi)

    def metrics(alpha, beta):
        tp, peak = shape(alpha, beta)
        t10 = crossing(alpha, beta, 0.1 * peak, 0.0, tp)
        t90 = crossing(alpha, beta, 0.9 * peak, 0.0, tp)
        th = crossing(alpha, beta, 0.5 * peak, tp, 50 * t_half + 10 * tp)
        # the tail crossing is decreasing: bisection above handles sign flips
        return 1.25 * (t90 - t10), th, peak

    alpha = math.log(2.0) / t_half
    beta = 2.5 / t_front
    for _ in range(60):
        # beta from the front time at fixed alpha (front shrinks as beta grows)
        lo, hi = beta / 8, beta * 8
        for _ in range(80):
            mid = math.sqrt(lo * hi)
            if metrics(alpha, mid)[0] > t_front:
                lo = mid
            else:
                hi = mid
        beta = math.sqrt(lo * hi)
        # alpha from the half-value time at fixed beta
        lo, hi = alpha / 4, alpha * 4
        for _ in range(80):
            mid = math.sqrt(lo * hi)
            if metrics(mid, beta)[1] > t_half:
                lo = mid
            else:
                hi = mid
        alpha = math.sqrt(lo * hi)
    _, _, peak = metrics(alpha, beta)
    return alpha, beta, 1.0 / peak


def double_exponential(t, i0, alpha, beta, k):
    return i0 * k * (np.exp(-alpha * t) - np.exp(-beta * t))


def heidler(t, i0, tau1, tau2, n, eta=None, t0=0.0):
    """Heidler lightning-current function (Heidler and Cvetic, the waveform
    class the paper's lightning examples use), started at t0:
    i(t) = (i0 / eta) s^n / (1 + s^n) exp(-(t - t0)/tau2), s = (t - t0)/tau1,
    for t > t0; eta None: the peak correction
    exp(-(tau1/tau2) (n tau2/tau1)^(1/n)), which makes the peak about i0."""
    t = np.asarray(t, dtype=np.float64) - t0
    if eta is None:
        eta = math.exp(-(tau1 / tau2) * (n * tau2 / tau1) ** (1.0 / n))
    x = np.where(t > 0, t / tau1, 0.0) ** n
    return np.where(t > 0, i0 / eta * x / (1.0 + x) * np.exp(-np.maximum(t, 0.0) / tau2), 0.0)


def ramp(t, i0, t_rise):
    """linear rise 0 -> i0 over t_rise, then flat"""
    return i0 * np.clip(t / t_rise, 0.0, 1.0)


# ---- material maps --------------------------------------------------------
def paint_blocks(n, blocks, background=0):
    """Material map from axis-aligned blocks of cells [(lo, hi, id)] with
    lo/hi = (i, j, k) half-open; later blocks override earlier ones."""
    nx, ny, nz = n
    cm = np.full((nz, ny, nx), background, dtype=np.uint8)
    for lo, hi, mid in blocks:
        cm[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] = mid
    return cm


def zero_walls(fields, n):
    """Zero tangential E on the low walls and normal H on the low walls, the
    entries a PEC box keeps at zero."""
    nx, ny, nz = n
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    masks = [(j == 0) | (k == 0), (i == 0) | (k == 0), (i == 0) | (j == 0), i == 0, j == 0, k == 0]
    for f, m in zip(fields, masks):
        f[m] = 0.0
    return fields


# ---- the configurations -----------------------------------------------------
def config1(n_steps=500):
    """48^3, dx = 0.1 m, PEC walls, soil (eps_r 10, sigma 0.01 S/m) in the
    lower half, Gaussian-derivative current (tau = 20 dt) on one Ez edge,
    three point E probes."""
    n = (48, 48, 48)
    dx, S = 0.1, 0.99
    cm = paint_blocks(n, [((0, 0, 0), (48, 48, 24), 1)])
    mats = [(1.0, 0.0, 1.0), (10.0, 0.01, 1.0)]
    dt = time_step(dx, S)
    tau = 20 * dt
    cur = gaussian_derivative(sample_times(n_steps, dx, S), tau, 6 * tau)
    return Scenario("config1_48cube_pec", n, dx, S, 0, cm, mats,
                    sources=[((24, 24, 28), 2, cur)],
                    probes=[(PROBE_E, (30, 24, 28), 2, 1), (PROBE_E, (24, 30, 20), 2, 1),
                            (PROBE_E, (12, 36, 30), 0, 1)],
                    n_steps=n_steps)


def config2(n_steps=4000, n=256):
    """256^3, dx = 0.5 m, 10-cell CPML; soil (eps_r 15, sigma 0.002) below
    node k = n/2; vertical thin wire r = 5 mm, 30 m, base-fed by a 1.2/50 us
    double exponential of 10 kA peak; probes: source-gap voltage and the wire
    current at five heights.  `n` < 256 gives the same layout scaled down
    (wire length capped to fit) for short parity runs."""
    dx, S = 0.5, 0.99
    nn = (n, n, n)
    c = n // 2
    cm = paint_blocks(nn, [((0, 0, 0), (n, n, c), 1)])
    mats = [(1.0, 0.0, 1.0), (15.0, 0.002, 1.0)]
    top = min(c + 61, n - 10 - 2)
    alpha, beta, k = double_exponential_params(1.2e-6, 50e-6)
    cur = double_exponential(sample_times(n_steps, dx, S), 10e3, alpha, beta, k)
    heights = [h for h in (c + 1, c + 16, c + 31, c + 46, c + 60) if h < top]
    probes = [(PROBE_V, (c, c, c), 2, 1)] + [(PROBE_I, (c, c, h), 2, 1) for h in heights]
    return Scenario(f"config2_{n}cube_cpml10_wire", nn, dx, S, 10, cm, mats,
                    wires=[((c, c, c + 1), (c, c, top), 0.005)],
                    sources=[((c, c, c), 2, cur)],
                    probes=probes, n_steps=n_steps)


def config3(n_steps=8000, scale=1):
    """512x512x384, dx = 0.25 m, 12-cell CPML; air above node k = 256,
    layer 1 (eps_r 10, sigma 0.01) for cells 248..255, layer 2 (eps_r 30,
    sigma 1e-3) below; buried 8x8 thin-wire mesh (10 m spacing, r = 6 mm,
    0.5 m deep) with a 2.5 m down-conductor at (236, 236); current lead
    along +x with a one-cell source gap, voltage lead along +y with a
    one-cell probe gap, both running into the CPML (the layout of the
    paper's ground-potential-rise model file); 1 kA ramp, 0.5 us rise."""
    dx, S = 0.25, 0.99
    nx, ny, nz = 512 // scale, 512 // scale, 384 // scale
    d = max(4, 12 // scale)
    surf = 256 // scale
    cm = paint_blocks((nx, ny, nz), [((0, 0, 0), (nx, ny, surf), 2),
                                     ((0, 0, surf - 8 // scale), (nx, ny, surf), 1)])
    mats = [(1.0, 0.0, 1.0), (10.0, 0.01, 1.0), (30.0, 1e-3, 1.0)]
    a = 0.006
    kw = surf - max(1, 2 // scale)
    lines = [116 // scale + (40 // scale) * q for q in range(8)]
    wires = []
    for y in lines:
        wires.append(((lines[0], y, kw), (lines[-1], y, kw), a))
    for x in lines:
        wires.append(((x, lines[0], kw), (x, lines[-1], kw), a))
    r = 236 // scale
    top = kw + max(2, 10 // scale)
    wires.append(((r, r, kw), (r, r, top), a))
    wires.append(((r, r, top), (r + 2, r, top), 0.003))            # stub to the source gap
    wires.append(((r + 3, r, top), (nx - d, r, top), 0.003))       # current lead
    wires.append(((r, r, top), (r, r + 2, top), 0.003))            # stub to the probe gap
    wires.append(((r, r + 3, top), (r, ny - d, top), 0.003))       # voltage lead
    cur = ramp(sample_times(n_steps, dx, S), 1e3, 0.5e-6)
    return Scenario(f"config3_{nx}x{ny}x{nz}_cpml{d}_mesh", (nx, ny, nz), dx, S, d, cm, mats,
                    wires=wires, sources=[((r + 2, r, top), 0, cur)],
                    probes=[(PROBE_V, (r, r + 2, top), 1, 1), (PROBE_I, (r + 2, r, top), 0, 1)],
                    n_steps=n_steps)


# ---- random problems for parity tests ---------------------------------------
def random_fields(rng, n, scale_h=1.0 / 377.0):
    nx, ny, nz = n
    f = [rng.standard_normal((nz, ny, nx)).astype(np.float64) for _ in range(6)]
    for c in range(3, 6):
        f[c] *= scale_h
    return zero_walls(f, n)


def random_scenario(seed, n=(17, 17, 17), dx=0.1, courant=0.99, cpml=0, n_blocks=5, n_mat=4,
                    n_wires=2, n_sources=2, n_probes=8, n_steps=40, fields=True, current_scale=1.0):
    """Random blocky media, thin wires, sources, probes and (optionally)
    random initial fields, all from one seed."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = n
    blocks = []
    for _ in range(n_blocks):
        lo = [int(rng.integers(0, m)) for m in n]
        hi = [int(rng.integers(l + 1, m + 1)) for l, m in zip(lo, n)]
        blocks.append((tuple(lo), tuple(hi), int(rng.integers(0, n_mat))))
    cm = paint_blocks(n, blocks)
    mats = [(float(rng.uniform(1.0, 20.0)), float(10 ** rng.uniform(-4, 0)), float(rng.uniform(1.0, 2.0)))
            for _ in range(n_mat)]
    lo_in = cpml + 1
    wires = []
    for _ in range(n_wires):
        axis = int(rng.integers(0, 3))
        p0 = [int(rng.integers(lo_in, m - lo_in)) for m in n]
        length = int(rng.integers(1, max(2, n[axis] - lo_in - p0[axis])))
        p1 = list(p0)
        p1[axis] = min(p0[axis] + length, n[axis] - lo_in)
        if p1[axis] <= p0[axis]:
            continue
        wires.append((tuple(p0), tuple(p1), float(dx * rng.uniform(0.005, 0.2))))
    t = np.arange(n_steps)
    sources = []
    for _ in range(n_sources):
        axis = int(rng.integers(0, 3))
        node = [int(rng.integers(lo_in, m - lo_in)) for m in n]
        w = rng.uniform(0.05, 0.4)
        cur = current_scale * rng.uniform(0.5, 2.0) * np.sin(w * t + rng.uniform(0, 6)) * np.exp(-t / rng.uniform(10, 40))
        sources.append((tuple(node), axis, cur))
    probes = []
    for q in range(n_probes):
        kind = q % 4
        axis = int(rng.integers(0, 3))
        node = [int(rng.integers(1, m - 1)) for m in n]
        ne = 1
        if kind == PROBE_V:
            ne = int(rng.integers(1, max(2, n[axis] - node[axis])))
        probes.append((kind, tuple(node), axis, ne))
    sc = Scenario(f"random{seed}_{nx}x{ny}x{nz}", n, dx, courant, cpml, cm, mats, wires, sources, probes,
                  n_steps)
    if fields:
        sc.fields = random_fields(rng, n)
    return sc


def with_random_debye(sc, seed, materials=(1, 2), max_poles=4):
    """give some materials of a scenario random Debye poles: deps ~ U[1, 40],
    tau = dt x U[5, 200] (relaxation times from a few to hundreds of steps)"""
    rng = np.random.default_rng(seed)
    dt = time_step(sc.dx, sc.courant)
    sc.debye = {}
    for m in materials:
        if m >= len(sc.materials):
            continue
        n_p = int(rng.integers(1, max_poles + 1))
        sc.debye[m] = ([float(v) for v in rng.uniform(1.0, 40.0, n_p)],
                       [float(v) for v in dt * rng.uniform(5.0, 200.0, n_p)])
    return sc


# Four-term Debye fit of a measured soil (the paper's table of Debye
# parameters for its buried-wire ground-potential-rise measurement):
# eps_inf 16.381, sigma_0 2.684 mS/m, poles (deps, tau).
PAPER_SOIL = dict(eps_inf=16.381, sigma=2.684e-3,
                  deps=[92.103, 20.825, 374.768, 10.387], tau=[7.404e-6, 1.062e-6, 2.162e-5, 1.008e-8])


def debye_soil(n_steps=4000, n=256):
    """The 256^3 thin-wire workload (config2 layout) over a dispersive soil:
    the lower half is the four-pole Debye soil above, the upper half air."""
    sc = config2(n_steps=n_steps, n=n)
    sc.name = f"debye_soil_{n}"
    sc.materials = [sc.materials[0], (PAPER_SOIL["eps_inf"], PAPER_SOIL["sigma"], 1.0)]
    sc.debye = {1: (list(PAPER_SOIL["deps"]), list(PAPER_SOIL["tau"]))}
    return sc


# Four-term Debye fits of three soil layers (the paper's table of Debye
# parameters computed for its apparent-resistivity example): per layer
# (eps_inf, sigma_0 S/m, deps[4], tau[4] s), top to bottom.
PAPER_LAYERS = [
    (15.767, 5.0e-3, [839.441, 143.901, 66.971, 31.515], [3.096e-5, 4.068e-6, 7.217e-7, 9.141e-8]),
    (13.488, 2.5e-3, [593.525, 101.748, 47.348, 22.273], [3.096e-5, 4.066e-6, 7.212e-7, 9.132e-8]),
    (11.884, 1.25e-3, [419.744, 71.960, 33.494, 15.757], [3.097e-5, 4.069e-6, 7.218e-7, 9.140e-8]),
]


# the array model file's source function (Sec. 4.3): Heidler, tau1 0.37 us,
# tau2 14 us, i0 1 A, n 10, eta 1 (no peak correction), started at 0.185 us
ARRAY_HEIDLER = dict(i0=1.0, tau1=3.7e-7, tau2=1.4e-5, n=10, eta=1.0, t0=1.85e-7)


def three_layer_array(n_steps=3000):
    """The electrode-array example of the paper's apparent-resistivity
    section: a 5 x 5 x 4 m domain at dx = 0.05 m (100 x 100 x 80 cells),
    10-cell CPML, three 1 m Debye soil layers (PAPER_LAYERS, top layer
    against the surface at 3 m) under air; four vertical rods of radius 8 mm
    from 2.95 m to 3.15 m at (1, 1), (2, 1), (4, 3) and (4, 4) m; a current
    lead (r = 3 mm) from the first rod's top towards the second with a
    one-cell source gap at x = 1.45 m, and a voltage lead from the third rod
    towards the fourth with a one-cell probe gap at y = 3.45 m.  The source
    is the model file's Heidler pulse (ARRAY_HEIDLER), which starts at
    0.185 us, step 1941 of dt = 95.3 ps.  Probes: voltage across the probe
    gap, current in the source gap."""
    dx = 0.05
    n = (100, 100, 80)
    ks = 60                                       # surface node (3 m)
    cm = paint_blocks(n, [((0, 0, 0), (100, 100, 20), 3), ((0, 0, 20), (100, 100, 40), 2),
                          ((0, 0, 40), (100, 100, ks), 1)])
    mats = [(1.0, 0.0, 1.0)] + [(e, s, 1.0) for e, s, _, _ in PAPER_LAYERS]
    debye = {m + 1: (list(d), list(t)) for m, (_, _, d, t) in enumerate(PAPER_LAYERS)}
    kb, kt = ks - 1, ks + 3                       # rods: 2.95 m .. 3.15 m
    rod = 0.008
    lead = 0.003
    wires = [((20, 20, kb), (20, 20, kt), rod), ((40, 20, kb), (40, 20, kt), rod),
             ((80, 60, kb), (80, 60, kt), rod), ((80, 80, kb), (80, 80, kt), rod),
             ((20, 20, kt), (29, 20, kt), lead), ((30, 20, kt), (40, 20, kt), lead),
             ((80, 60, kt), (80, 69, kt), lead), ((80, 70, kt), (80, 80, kt), lead)]
    cur = heidler(sample_times(n_steps, dx, 0.99), **ARRAY_HEIDLER)
    sc = Scenario("three_layer_array", n, dx, 0.99, 10, cm, mats, wires=wires,
                  sources=[((29, 20, kt), 0, cur)],
                  probes=[(PROBE_V, (80, 69, kt), 1, 1), (PROBE_I, (29, 20, kt), 0, 1)],
                  n_steps=n_steps)
    sc.debye = debye
    return sc


# ---- grounding-electrode domains (the batched and surrogate workloads) -----
GROUND_DX = 0.25          # m; fixed so every domain spans the same time window
GROUND_CPML = 8
GROUND_STEPS = 2000
GROUND_SAMPLES = 512
LEAD_RADIUS = 0.003


def grounding_cells(length, depth):
    """(rod length, burial depth of its top) in cells of GROUND_DX: the
    discrete geometry the domain builder uses."""
    return max(1, int(round(length / GROUND_DX))), int(round(depth / GROUND_DX))


def grounding_domain(n, eps_r, sigma, length, radius, depth, rise, n_steps=GROUND_STEPS, name="ground",
                     incline=0.0, courant=0.99):
    """One grounding-electrode domain of n^3 cells, dx = 0.25 m, 8-cell CPML:
    soil (eps_r, sigma) below the surface node n - 14, air above; a vertical
    rod of the given length and radius whose top is `depth` m below the
    surface at the domain centre; a riser (same radius) up to 1 m above the
    surface; from its top a current lead along +x with a one-cell source gap
    two cells out and a voltage lead along +y with a one-cell probe gap two
    cells out, both running into the CPML (the layout of the paper's
    ground-potential-rise model file); a 1 kA linear ramp of the given rise
    time on the source gap.  Probes: gap voltage and source current.
    incline > 0 (rad from the vertical): the rod is an oblique wire of the
    same length leaning towards -x from the riser's bottom node, which joins
    it to the riser (run below the oblique wire's Courant limit)."""
    dx = GROUND_DX
    d = GROUND_CPML
    c = n // 2
    ks = n - 14                                    # surface node
    lc, dc = grounding_cells(length, depth)
    kd = ks - dc                                   # rod top node
    kb = kd - lc * math.cos(incline)               # rod bottom (node units)
    xb = c - lc * math.sin(incline)
    if kb < d + 2 or xb < d + 2:
        raise ValueError("rod does not fit the domain")
    kt = ks + 4                                    # riser top, 1 m above the surface
    cm = paint_blocks((n, n, n), [((0, 0, 0), (n, n, ks), 1)])
    mats = [(1.0, 0.0, 1.0), (float(eps_r), float(sigma), 1.0)]
    rod = [((c, c, kd - lc), (c, c, kd), radius)] if incline == 0 else []
    wires = rod + [((c, c, kd), (c, c, kt), radius),     # riser
             ((c, c, kt), (c + 2, c, kt), LEAD_RADIUS),
             ((c + 3, c, kt), (n - d, c, kt), LEAD_RADIUS),
             ((c, c, kt), (c, c + 2, kt), LEAD_RADIUS),
             ((c, c + 3, kt), (c, n - d, kt), LEAD_RADIUS)]
    cur = ramp(sample_times(n_steps, dx, courant), 1e3, rise)
    sc = Scenario(name, (n, n, n), dx, courant, d, cm, mats, wires=wires,
                  sources=[((c + 2, c, kt), 0, cur)],
                  probes=[(PROBE_V, (c, c + 2, kt), 1, 1), (PROBE_I, (c + 2, c, kt), 0, 1)],
                  n_steps=n_steps)
    if incline != 0:
        sc.owires = [((float(c), float(c), float(kd)), (xb, float(c), kb), radius)]
    return sc


def config4(n_domains=256, seed=0, n_steps=GROUND_STEPS, n_range=(48, 128)):
    """The batched workload: n_domains rods, side ~ U{48..128} cells,
    eps_r ~ U[4, 40], log10 sigma ~ U[-4, -1], r = 8 mm at the surface,
    L ~ U[1, min(10, 0.25 (N - 28))] m, 1 kA ramp of 0.25 us rise."""
    rng = np.random.default_rng(seed)
    out = []
    for q in range(n_domains):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        eps = float(rng.uniform(4.0, 40.0))
        sig = float(10 ** rng.uniform(-4.0, -1.0))
        lmax = min(10.0, GROUND_DX * (n - 28))
        length = float(rng.uniform(1.0, lmax))
        out.append(grounding_domain(n, eps, sig, length, 0.008, 0.0, 0.25e-6, n_steps, name=f"rod{q}_n{n}"))
    return out


INCLINED_COURANT = 0.95   # below the 8 mm oblique rod's Courant limit (about 0.978 at dx 0.25 m)


def config4_inclined(n_domains=256, seed=0, n_steps=GROUND_STEPS, n_range=(48, 128)):
    """The batched workload with inclined rods: as config4, each rod leaning
    at U[15, 60] degrees from the vertical (an oblique wire joined to the
    riser), L capped so it stays inside the domain; Courant number 0.95."""
    rng = np.random.default_rng(seed)
    out = []
    for q in range(n_domains):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        eps = float(rng.uniform(4.0, 40.0))
        sig = float(10 ** rng.uniform(-4.0, -1.0))
        th = math.radians(float(rng.uniform(15.0, 60.0)))
        lmax = min(10.0, GROUND_DX * (n - 28), GROUND_DX * (n // 2 - 11) / math.sin(th))
        length = float(rng.uniform(1.0, lmax))
        out.append(grounding_domain(n, eps, sig, length, 0.008, 0.0, 0.25e-6, n_steps, name=f"incl{q}_n{n}",
                                    incline=th, courant=INCLINED_COURANT))
    return out


SURROGATE_N = 64          # domain side used for the surrogate's runs


def surrogate_inputs(seed):
    """The six surrogate parameters of one seeded run: eps_r ~ U[4, 40],
    log10 sigma ~ U[-4, -1], rod length (m), radius ~ U[4, 16] mm, burial
    depth of the rod top ~ U[0, 1] m, rise time ~ U[0.1, 0.5] us; the length
    is drawn from U[1, Lmax - depth] with Lmax the config-4 cap of the
    64-cell domain."""
    rng = np.random.default_rng(seed)
    eps = float(rng.uniform(4.0, 40.0))
    lsig = float(rng.uniform(-4.0, -1.0))
    radius = float(rng.uniform(0.004, 0.016))
    depth = float(rng.uniform(0.0, 1.0))
    rise = float(rng.uniform(0.1e-6, 0.5e-6))
    lmax = min(10.0, GROUND_DX * (SURROGATE_N - 28)) - depth
    length = float(rng.uniform(1.0, lmax))
    return np.array([eps, lsig, length, radius, depth, rise])


def surrogate_domain(params, n_steps=GROUND_STEPS):
    eps, lsig, length, radius, depth, rise = [float(v) for v in params]
    return grounding_domain(SURROGATE_N, eps, 10 ** lsig, length, radius, depth, rise, n_steps)


def impedance_waveform(v_gap, dt, n_samples=GROUND_SAMPLES, i_peak=1e3):
    """Output of a grounding run: the gap voltage (sampled at t_{n+1}) over
    the peak current, linearly interpolated to n_samples uniform instants of
    [0, n_steps dt]."""
    v = np.asarray(v_gap, dtype=np.float64)
    t_src = (np.arange(len(v)) + 1.0) * dt
    t = np.linspace(0.0, len(v) * dt, n_samples)
    return np.interp(t, np.concatenate([[0.0], t_src]), np.concatenate([[0.0], v])) / i_peak


# ---- lightning strike to a lattice tower -----------------------------------
TOWER_DX = 0.5
TOWER_RADIUS = 0.02
TOWER_CHANNEL_OHM = 400.0


def tower_members(x0=36, y0=36, zs=20):
    """Members of a synthetic 30 m lattice tower (node coordinates, all
    integer so both wire models can draw them): four legs rising from a
    6 m square at the soil surface (node plane zs) to a 2 m square at 24 m,
    a vertical 2 m square section to 30 m with a frame at 28 m, a pyramid
    peak 2 m above it, V-shaped cross-arms at 28 m reaching 7 m out on both
    sides along x, and 3 m ground rods under the legs."""
    m = []
    corners = [(-1, -1), (1, -1), (1, 1), (-1, 1)]
    for sx, sy in corners:
        base = (x0 + 6 * sx, y0 + 6 * sy, zs)
        waist = (x0 + 2 * sx, y0 + 2 * sy, zs + 48)
        top = (x0 + 2 * sx, y0 + 2 * sy, zs + 60)
        m += [(base, waist), (waist, top), (top, (x0, y0, zs + 64)), ((base[0], base[1], zs - 6), base)]
    for q in range(4):
        a, b = corners[q], corners[(q + 1) % 4]
        m.append(((x0 + 2 * a[0], y0 + 2 * a[1], zs + 56), (x0 + 2 * b[0], y0 + 2 * b[1], zs + 56)))
    for sx in (-1, 1):
        tip = (x0 + 16 * sx, y0, zs + 56)
        for sy in (-1, 1):
            m.append(((x0 + 2 * sx, y0 + 2 * sy, zs + 56), tip))
    return m


def lightning_tower(model="oblique", n_steps=3000, i0=10e3, n=(72, 72, 100)):
    """Direct strike to a lattice tower over lossy soil (the lightning
    overvoltage example of the paper, with a synthetic tower): soil eps_r 10,
    sigma 2 mS/m below the node plane 20, 10-cell CPML, dx = 0.5 m, the tower
    at the centre of the n[0] x n[1] plan (72 x 72 x 100 cells by default); the tower
    of tower_members() in the oblique wire model or as staircase wires; a
    phase conductor along y 2 m below the +x arm tip (axis-aligned thin wire
    in both cases, into the CPML); a vertical lightning channel from the
    peak into the CPML driven, across its lowest cell, by 400 ohm x a
    Heidler current (10 kA, 1.2 / 50 us class) behind 400 ohm; probes: the
    grid voltage across the insulator (phase conductor up to the arm tip),
    the current in the channel's lowest cell and, for oblique wires, the
    arm tip's in-cell potential (the insulator voltage is the sum of the
    first and the last).  Courant 0.93 (below the oblique members' limit,
    used for both models)."""
    nx, ny, nz = n
    x0, y0, zs = nx // 2, ny // 2, 20
    cm = np.zeros((nz, ny, nx), np.uint8)
    cm[:zs] = 1
    mats = [(1.0, 0.0, 1.0), (10.0, 2e-3, 1.0)]
    sc = Scenario(f"lightning_tower_{model}", n, TOWER_DX, 0.93, 10, cm, mats, n_steps=n_steps)
    dt = sc.courant * TOWER_DX / (C0 * math.sqrt(3.0))
    t = (np.arange(n_steps) + 0.5) * dt
    emf = TOWER_CHANNEL_OHM * heidler(t, i0, 0.3e-6, 50e-6, 4)
    peak = (x0, y0, zs + 64)
    tip = (x0 + 16, y0, zs + 56)
    members = tower_members(x0, y0, zs)
    if model == "oblique":
        sc.owires = [(p, q, TOWER_RADIUS) for p, q in members]
        ch = len(sc.owires)
        sc.owires.append((peak, (x0, y0, nz - 5), TOWER_RADIUS))
        sc.owire_sources = [(ch, 0, emf, TOWER_CHANNEL_OHM)]
        sc.owire_probes = [(ch, 0), tip]          # channel current; the arm tip's in-cell potential
    elif model == "staircase":
        sc.wire_paths = [(p, q, TOWER_RADIUS) for p, q in members]
        sc.wires = [((x0, y0, zs + 65), (x0, y0, nz - 5), TOWER_RADIUS)]
        sc.vsources = [((x0, y0, zs + 64), 2, emf, TOWER_CHANNEL_OHM)]
        sc.probes = [(1, (x0, y0, zs + 64), 2, 1)]
    else:
        raise ValueError(model)
    sc.wires = list(sc.wires) + [((tip[0], 2, tip[2] - 4), (tip[0], ny - 2, tip[2] - 4), 0.01)]
    sc.probes = [(0, (tip[0], y0, tip[2] - 4), 2, 4)] + list(sc.probes)
    return sc
