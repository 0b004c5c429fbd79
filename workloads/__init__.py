"""Seeded synthetic inputs for the absorbing-layer lattice Boltzmann workloads.

This module only draws and lays out INPUTS: lattice sizes, relaxation rates,
absorbing-strength profiles, initial density fields, request traces.  It holds
none of the scheme's arithmetic, and both the CUDA path (through the tests and
``bench.py``) and the CPU oracle consume what it returns.

The inputs stand in for the paper's 2-D acoustic-pulse experiment (Sec. 4.1,
Eqs. pulseprofile, 3:para0): a Gaussian density pulse of amplitude eps and
half-width b on a uniform medium at rest or in uniform mean flow, with the
populations at equilibrium and an absorbing layer on the four sides.  The
paper's own figure data is not available, so every field here is synthetic and
seeded with ``numpy.random.default_rng(seed)``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

CS = 1.0 / math.sqrt(3.0)
VARIANT_CYCLE = ("I", "II", "III")


def rate_from_viscosity(nu: float) -> float:
    """Relaxation rate s with nu = c_s^2 (1/s - 1/2) (delta t = 1), Sec. 2.2.2."""
    return 1.0 / (3.0 * nu + 0.5)


def bgk_rates(s: float) -> np.ndarray:
    """All nine rates equal (the paper's BGK setting; the conserved rows use s_c = s)."""
    return np.full(9, float(s))


def layer_depth(n: int, width: int) -> np.ndarray:
    """Depth d of each index in an absorbing layer of `width` cells at both ends of an
    axis of n cells: d = width - min(i, n-1-i), clamped to [0, width]; the outermost
    cell has d = width."""
    i = np.arange(n)
    d = width - np.minimum(i, n - 1 - i)
    return np.clip(d, 0, width).astype(np.float64)


def ramp_profile(n: int, width: int, chi_max: float, power: float = 2.0) -> np.ndarray:
    """chi(d) = chi_max (d / width)^power: Table tab:sigma's second profile with
    eta = chi_max (power 2 is the quadratic ramp of the workloads)."""
    if width <= 0 or chi_max == 0.0:
        return np.zeros(n)
    return chi_max * (layer_depth(n, width) / width) ** power


def viscous_ramp(n: int, width: int) -> np.ndarray:
    """Layer fraction r = d / width in [0, 1] for the viscosity sponge of Sec. 4.1
    (the relaxation frequency falls linearly from its physical value at the
    inner edge of the layer, r = 0, to 1 at the wall, r = 1)."""
    if width <= 0:
        return np.zeros(n)
    return layer_depth(n, width) / width


def polynomial_profile(n: int, width: int, A: float, power: int = 4) -> np.ndarray:
    """Table tab:sigma's polynomial profile,
    sigma(x) = A (x - x0)^power (L - x) (power + 1)(power + 2) / (L - x0)^(power + 2),
    laid across the layer as orszag_profile lays its own (x0 at depth 0, L at depth
    width + 1).  A is the profile's integral over [x0, L]: the Beta integral of
    t^power (1 - t) is 1 / ((power + 1)(power + 2)).  With power = 4,
    orszag_profile(chi) is this profile with A = chi (L - x0) 3125 / (256 * 30):
    A is an integral over the layer, chi the peak of the normalised profile."""
    if width <= 0:
        return np.zeros(n)
    d = layer_depth(n, width)
    L = width + 1.0
    sig = A * d**power * (L - d) * (power + 1) * (power + 2) / L ** (power + 2)
    return np.where(d > 0, sig, 0.0)


def orszag_profile(n: int, width: int, chi: float) -> np.ndarray:
    """sigma = chi * sigma~ with the normalised A = n = 4 profile of
    Eq. (normalizedsigma), sigma~(x) = 3125 (L - x)(x - x0)^4 / (256 (L - x0)^5),
    laid across the layer with x0 at the inner edge (depth 0) and L one cell
    beyond the outermost cell (depth width + 1), so sigma~ peaks at 1 at 80 % of
    the way through."""
    if width <= 0:
        return np.zeros(n)
    d = layer_depth(n, width)
    L = width + 1.0
    sig = 3125.0 * (L - d) * d**4 / (256.0 * L**5)
    return chi * np.where(d > 0, sig, 0.0)


def outflow_layer(n: int, width: int, chi: float, profile: str = "orszag") -> np.ndarray:
    """Absorbing strength along x for the channel of Sec. 4.2: a layer of `width`
    cells at the right (outflow) end only, depth 0 at its inner edge rising to
    `width` at the last cell; profile "orszag" (Eq. normalizedsigma, A = n = 4),
    "ramp" (quadratic) or "viscous" (the layer fraction r = d / width)."""
    out = np.zeros(n)
    if width <= 0:
        return out
    i = np.arange(n)
    d = np.clip(i - (n - 1 - width), 0, width).astype(np.float64)
    if profile == "orszag":
        L = width + 1.0
        out = chi * np.where(d > 0, 3125.0 * (L - d) * d**4 / (256.0 * L**5), 0.0)
    elif profile == "ramp":
        out = chi * (d / width) ** 2
    elif profile == "viscous":
        out = d / width
    else:
        raise ValueError(profile)
    return out


def gaussian_pulse(nx: int, ny: int, x0: float, y0: float, eps: float, b: float) -> np.ndarray:
    """rho' = eps exp(-alpha r^2), alpha = ln2 / b^2 (Eq. 3:para0), on cell centres
    (ix, iy), as [ny, nx]."""
    alpha = math.log(2.0) / (b * b)
    x = np.arange(nx, dtype=np.float64)[None, :]
    y = np.arange(ny, dtype=np.float64)[:, None]
    return eps * np.exp(-alpha * ((x - x0) ** 2 + (y - y0) ** 2))


@dataclass
class Workload:
    """One lattice problem: sizes, rates, damping, boundary, initial fields, steps."""

    name: str
    nx: int
    ny: int
    s: np.ndarray
    variant: str = "II"
    bc: str = "dirichlet"
    n: float = 0.5
    m: float = 0.5
    rho0: float = 1.0
    u0: tuple = (0.0, 0.0)
    rho_f: float = 1.0
    u_f: tuple = (0.0, 0.0)
    chi_x: np.ndarray = None
    chi_y: np.ndarray = None
    rho_dev: np.ndarray = None  # initial rho - rho0, [ny, nx]
    steps: int = 100
    storage: str = "f32"
    width: int = 0
    chi_max: float = 0.0
    seed: int | None = None
    meta: dict = field(default_factory=dict)
    source: tuple = (0.0, 0.0, 0.0)  # channel: (amplitude, omega per step, phase) of the line source

    def __post_init__(self):
        if self.chi_x is None:
            self.chi_x = np.zeros(self.nx)
        if self.chi_y is None:
            self.chi_y = np.zeros(self.ny)

    @property
    def cells(self) -> int:
        return self.nx * self.ny

    def density_deviation(self) -> np.ndarray:
        """Initial rho - rho0, [ny, nx]: the stored field, else the Gaussian pulse
        described by meta (eps, b, x0, y0), else zero.  Built on demand so that
        long request traces stay small."""
        if self.rho_dev is not None:
            return self.rho_dev
        mt = self.meta
        if mt.get("eps", 0.0) != 0.0:
            return gaussian_pulse(self.nx, self.ny, mt["x0"], mt["y0"], mt["eps"], mt["b"])
        return np.zeros((self.ny, self.nx))

    def initial_fields(self):
        """(rho, u_x, u_y) of the initial state, [ny, nx] FP64 each."""
        rho = self.rho0 + self.density_deviation()
        return rho, np.full_like(rho, self.u0[0]), np.full_like(rho, self.u0[1])

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)


def pulse_workload(nx=100, ny=100, variant="II", storage="f32", nu=1e-3, eps=1e-3, b=3.0,
                   x0=None, y0=None, width=20, chi_max=0.1, steps=300, u0=(0.0, 0.0),
                   bc="dirichlet", name="pulse", power=2.0) -> Workload:
    """Gaussian pulse on a uniform medium with a ramped absorbing layer on all sides,
    q_ref = the far-field state."""
    x0 = (nx - 1) / 2.0 if x0 is None else x0
    y0 = (ny - 1) / 2.0 if y0 is None else y0
    return Workload(
        name=name, nx=nx, ny=ny, s=bgk_rates(rate_from_viscosity(nu)), variant=variant, bc=bc,
        u0=tuple(u0), u_f=tuple(u0), chi_x=ramp_profile(nx, width, chi_max, power),
        chi_y=ramp_profile(ny, width, chi_max, power),
        steps=steps, storage=storage,
        width=width, chi_max=chi_max, meta={"eps": eps, "b": b, "x0": x0, "y0": y0, "nu": nu},
    )


def small_pulse(variant="II", storage="f64") -> Workload:
    """100 x 100 lattice, rho0 = 1, u0 = 0, nu = 1e-3, Gaussian pulse eps = 1e-3, b = 3
    at the centre, layer of 20 cells with chi(d) = 0.1 (d/20)^2, q_ref at rest, 300 steps."""
    return pulse_workload(100, 100, variant=variant, storage=storage, name="pulse-100x100")


def chi_sweep(storage="f64", steps=300) -> list:
    """The 100 x 100 pulse geometry (20-cell quadratic ramp, type II) with the peak
    strength swept toward the critical value of Eq. criticalchi: chi_max = 0.1, 0.5,
    1.0, 1.5, 1.9 and 4/s - 0.001 (the choice of Sec. 4.1), s = 1/(3 nu + 1/2)."""
    base = pulse_workload(100, 100, variant="II", storage=storage, steps=steps,
                          name="chi-sweep-100x100")
    s = float(base.s[0])
    out = []
    for cm in (0.1, 0.5, 1.0, 1.5, 1.9, 4.0 / s - 0.001):
        prof = ramp_profile(100, base.width, cm)
        out.append(base.with_(chi_x=prof, chi_y=prof.copy(), chi_max=cm))
    return out


CHI_MAX_CHOICES = (0.01, 0.05, 0.2, 1.0)


def mean_flow_pulse(seed: int = 0, variant="II", storage="f32", side=1024, steps=5000) -> Workload:
    """side^2 lattice (default 1024^2), uniform mean flow Mach 0.2 along x
    (u0 = 0.2/sqrt(3)), pulse eps = 1e-3, b = 5 at a seeded interior point outside the
    layer, layer width 64, chi_max drawn from {0.01, 0.05, 0.2, 1.0}, quadratic ramp."""
    rng = np.random.default_rng(seed)
    width = 64
    chi_max = float(rng.choice(CHI_MAX_CHOICES))
    lo, hi = width + 10, side - width - 10
    x0 = float(rng.uniform(lo, hi))
    y0 = float(rng.uniform(lo, hi))
    u = 0.2 * CS
    w = pulse_workload(side, side, variant=variant, storage=storage, eps=1e-3, b=5.0, x0=x0, y0=y0,
                       width=width, chi_max=chi_max, steps=steps, u0=(u, 0.0),
                       name=f"mean-flow-pulse-{side}x{side}")
    w.seed = seed
    return w


def quiescent(side: int, storage="f32", steps=200, width=128, chi_max=0.1, variant="II",
              pulse: bool = False) -> Workload:
    """Square lattice at rest with a 128-cell ramped layer (the roofline sweep). With
    pulse=True a centred eps = 1e-3, b = 5 pulse is added for error measurements."""
    w = pulse_workload(side, side, variant=variant, storage=storage, eps=1e-3 if pulse else 0.0,
                       b=5.0, width=width, chi_max=chi_max, steps=steps,
                       name=f"quiescent-{side}x{side}")
    return w


def line_source(nx: int = 800, ny: int = 200, variant: str = "II", width: int = 160,
                amplitude: float = 1e-3, period: float = 100.0, u0=(0.0, 0.0), nu: float = 2e-4,
                steps: int | None = None, storage: str = "f32", profile: str | None = None,
                eps: float = 1e-3, name: str = "line-source") -> Workload:
    """The time-dependent acoustic line source of Sec. 4.2 in lattice units: a
    channel W = 4H with H = ny cells (200 cells per unit length), periodic in y,
    the source rho0 + A sin(2 pi t / period) on the left edge, an outflow on the
    right, and an absorbing layer of `width` cells (0.8 H) in front of the
    outflow with chi_max = 4/s - eps (the paper's choice).  omega = 2 per unit
    time with delta t = 1/200 gives a period of 100 steps and a wavelength of
    c_s * 100 = 57.7 cells (c_s / 2 = 0.2887 units).  nu = 2e-4 is Re = 1/nu
    = 1e6 in those units.  The default number of steps is the paper's sample
    time T_o + 10 T_p (T_o = W / (c_s + u0x), T_p = one period)."""
    s = rate_from_viscosity(nu)
    chi_max = 4.0 / s - eps
    if profile is None:
        profile = "viscous" if variant == "viscous" else "orszag"
    chi_x = outflow_layer(nx, width, chi_max, profile) if variant != "none" else np.zeros(nx)
    if steps is None:
        steps = int(round(nx / (CS + u0[0]) + 10 * period))
    return Workload(name=name, nx=nx, ny=ny, s=np.full(9, s), variant=variant, bc="channel",
                    u0=tuple(u0), u_f=tuple(u0), chi_x=chi_x, chi_y=np.zeros(ny), steps=steps,
                    storage=storage, width=width, chi_max=chi_max,
                    source=(amplitude, 2.0 * math.pi / period, 0.0),
                    meta={"period": period, "wavelength": (CS + u0[0]) * period})


@dataclass
class Workload3:
    """A D3Q15 lattice problem: sizes, rates (15, row order of M), damping,
    per-axis strengths, far field, reference state, initial density deviation
    (u = u0 everywhere) and step count."""
    name: str
    nx: int
    ny: int
    nz: int
    s: np.ndarray
    variant: str
    chi_x: np.ndarray
    chi_y: np.ndarray
    chi_z: np.ndarray
    rho_dev: np.ndarray
    steps: int
    bc: str = "dirichlet"
    n: float = 0.5
    m: float = 0.5
    rho0: float = 1.0
    u0: tuple = (0.0, 0.0, 0.0)
    rho_f: float = 1.0
    u_f: tuple = (0.0, 0.0, 0.0)
    storage: str = "f32"

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz


def pulse3d(side: int = 256, storage: str = "f32", steps: int = 100, width: int = 16,
            chi_max: float = 0.1, variant: str = "II", eps: float = 1e-3, b: float = 5.0,
            nu: float = 1e-3, u0=(0.0, 0.0, 0.0), ny: int | None = None,
            nz: int | None = None) -> Workload3:
    """The acoustic pulse of Sec. 4.1 in three dimensions: a Gaussian density
    pulse (eps, half width b) at the centre of a side^3 box (ny, nz override the
    other sides) with a quadratic ramp layer of `width` cells on every face,
    rates of viscosity nu, Dirichlet far field."""
    ny = side if ny is None else ny
    nz = side if nz is None else nz
    s = rate_from_viscosity(nu)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(side), indexing="ij")
    r2 = (x - (side - 1) / 2) ** 2 + (y - (ny - 1) / 2) ** 2 + (z - (nz - 1) / 2) ** 2
    return Workload3(name=f"pulse3d-{side}x{ny}x{nz}", nx=side, ny=ny, nz=nz, s=np.full(15, s),
                     variant=variant, chi_x=ramp_profile(side, width, chi_max),
                     chi_y=ramp_profile(ny, width, chi_max), chi_z=ramp_profile(nz, width, chi_max),
                     rho_dev=eps * np.exp(-math.log(2.0) * r2 / b**2), steps=steps,
                     storage=storage, u0=tuple(u0), u_f=tuple(u0))


def stability_map(s_values=(1.9, 1.99, 1.999), bulk=(1.0, 1.5, None), heat=(1.2, 1.8, None),
                  u_values=(0.0, 0.05, 0.1, 0.15, 0.2),
                  thetas=(0.0, math.pi / 8, math.pi / 4), variants=("I", "II", "III"),
                  n: float = 0.5, m: float = 0.5):
    """Cases of the stability map: Sec. 3.3's Von Neumann study extended to
    distinct MRT rates.  For each shear rate s (s_nu = s_c = s), bulk rate
    s_e = s_eps in `bulk` and heat-flux rate s_q in `heat` (None: equal to s),
    target flow u^f = (U, 0), wave direction theta and damping variant, one
    record [s_0..s_8, n, m, u_x, u_y, theta, chi = 0] in the row order of M.
    Returns (variants, cases[N, 15])."""
    vs, cases = [], []
    for v in variants:
        for s in s_values:
            for se in bulk:
                for sq in heat:
                    se_ = s if se is None else se
                    sq_ = s if sq is None else sq
                    s9 = [s, s, s, se_, se_, sq_, sq_, s, s]
                    for u in u_values:
                        for th in thetas:
                            vs.append(v)
                            cases.append(s9 + [n, m, u, 0.0, th, 0.0])
    return vs, np.array(cases, dtype=np.float64)


def batch_of_lattices(seed: int = 0, count: int = 256, lo: int = 64, hi: int = 1024,
                      steps: int = 1000, storage="f32") -> list[Workload]:
    """`count` independent lattices: sides log-uniform in [lo, hi] per axis, seeded pulse
    location, Mach in [0, 0.2], chi_max log-uniform in [1e-3, 1], layer width uniform in
    [8, 64], damping variant cycled I, II, III."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        nx = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        ny = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        mach = float(rng.uniform(0.0, 0.2))
        chi_max = float(math.exp(rng.uniform(math.log(1e-3), math.log(1.0))))
        width = int(rng.integers(8, 65))
        width = min(width, (min(nx, ny) - 2) // 2)
        x0 = float(rng.uniform(0.25 * nx, 0.75 * nx))
        y0 = float(rng.uniform(0.25 * ny, 0.75 * ny))
        variant = VARIANT_CYCLE[k % 3]
        w = pulse_workload(nx, ny, variant=variant, storage=storage, eps=1e-3, b=5.0, x0=x0, y0=y0,
                           width=width, chi_max=chi_max, steps=steps, u0=(mach * CS, 0.0),
                           name=f"batch-{k}")
        w.seed = seed
        out.append(w)
    return out


@dataclass
class Request:
    arrival: float
    workload: Workload


def request_trace(seed: int = 0, rate: float = 200.0, duration: float = 60.0, lo: int = 128,
                  hi: int = 4096, steps_lo: int = 500, steps_hi: int = 5000,
                  storages=("f32", "f16dev"), max_requests: int | None = None) -> list[Request]:
    """Poisson arrivals (rate per second) of sweep jobs: square side log-uniform in
    [lo, hi], steps uniform in [steps_lo, steps_hi], chi_max / width / variant drawn as in
    batch_of_lattices, storage drawn from `storages`."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    k = 0
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t >= duration or (max_requests is not None and len(out) >= max_requests):
            break
        side = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        steps = int(rng.integers(steps_lo, steps_hi + 1))
        mach = float(rng.uniform(0.0, 0.2))
        chi_max = float(math.exp(rng.uniform(math.log(1e-3), math.log(1.0))))
        width = min(int(rng.integers(8, 65)), (side - 2) // 2)
        x0 = float(rng.uniform(0.25 * side, 0.75 * side))
        y0 = float(rng.uniform(0.25 * side, 0.75 * side))
        storage = storages[int(rng.integers(0, len(storages)))]
        w = pulse_workload(side, side, variant=VARIANT_CYCLE[k % 3], storage=storage, eps=1e-3,
                           b=5.0, x0=x0, y0=y0, width=width, chi_max=chi_max, steps=steps,
                           u0=(mach * CS, 0.0), name=f"req-{k}")
        w.seed = seed
        out.append(Request(arrival=t, workload=w))
        k += 1
    return out
