"""Seeded synthetic inputs for the thermal pseudopotential LB workloads.

This module holds only the input recipes (initial density and temperature
fields, parameter draws).  It contains none of the method's arithmetic, so
both the CUDA path and the CPU oracle can be fed from it.

Random numbers come from SplitMix64 (Steele, Lea & Flood, OOPSLA 2014), a
counter-based generator: the value for site index s under seed k is
SplitMix64(SplitMix64(k) XOR s), mapped to a 53-bit double in [0, 1).
The same seed therefore gives the same field on every machine.

Workload recipes (all periodic D2Q9 lattices, Carnahan-Starling EOS with
a = 1, b = 4, R = 1, G = -1):

* ``slab_64``      64 x 64, T = 0.85 T_c, liquid slab x in [nx/2-16, nx/2+16)
                   at rho_l = 0.35 in vapour rho_g = 0.03, noise +-1e-3 (seed 1)
* ``droplet_512``  512 x 512, droplet radius 64 at rho_l in rho_g, T linear
                   in x from 0.80 T_c to 0.90 T_c
* ``spinodal_4096`` 4096 x 4096, T = 0.75 T_c, rho = 0.12 + noise +-0.01 (seed 3)
* ``batched_sweep`` 256 domains, side L ~ U{64..512}, T/T_c ~ U[0.6, 0.95],
                   G ~ U[-1.2, -0.8], tau_f ~ U[0.6, 1.2], droplet or slab
"""
from __future__ import annotations

import dataclasses

import numpy as np

#: Critical temperature and density of the Carnahan-Starling EOS with
#: a = 1, b = 4, R = 1 (the point where dp/drho = d2p/drho2 = 0; the tests
#: check these constants against an independent high-precision solve).
CS_TC = 0.09432870313855984
CS_RHOC = 0.130443

RHO_LIQUID = 0.35
RHO_GAS = 0.03

#: Liquid-vapour coexistence of the Carnahan-Starling EOS (a = 1, b = 4,
#: R = 1) by Maxwell's equal-area construction: (T/T_c, rho_g, rho_l).
#: Written by ``python -m oracle.coexistence``; the seeded sweep starts each
#: droplet or slab at these densities.
COEXISTENCE_CS = (
    (0.60, 0.003081458539929346, 0.40620413975436337),
    (0.61, 0.0034997542027268625, 0.4014427889164023),
    (0.62, 0.003957347577293854, 0.39667751203982027),
    (0.63, 0.004456311234053168, 0.3919060639255548),
    (0.64, 0.004998765384390647, 0.38712614902380965),
    (0.65, 0.005586886973241947, 0.3823354103809645),
    (0.66, 0.0062229202616471595, 0.3775314175849033),
    (0.67, 0.006909189021726869, 0.3727116535129428),
    (0.68, 0.007648110510058689, 0.36787349965044014),
    (0.69, 0.008442211437681275, 0.36301421970323666),
    (0.70, 0.009294146218119775, 0.35813094117095823),
    (0.71, 0.010206717851948169, 0.3532206344776867),
    (0.72, 0.011182901901625615, 0.34828008916736725),
    (0.73, 0.012225874129302991, 0.34330588655791816),
    (0.74, 0.013339042520686866, 0.3382943681025933),
    (0.75, 0.014526084610435294, 0.3332415985191704),
    (0.76, 0.015790991273582196, 0.328143322502446),
    (0.77, 0.01713811847365384, 0.3229949135127225),
    (0.78, 0.018572248890532, 0.3177913127035731),
    (0.79, 0.020098665931519172, 0.3125269554742717),
    (0.80, 0.021723243418436067, 0.3071956823451157),
    (0.81, 0.023452555332236853, 0.30179062976703364),
    (0.82, 0.025294011520760037, 0.2963040949543186),
    (0.83, 0.02725602744411192, 0.2907273666617526),
    (0.84, 0.029348239174172765, 0.28505051068649256),
    (0.85, 0.031581779506976666, 0.27926209423373366),
    (0.86, 0.03396963805744112, 0.2733488262751818),
    (0.87, 0.03652713905616116, 0.2672950801797546),
    (0.88, 0.03927258783124093, 0.26108224763314025),
    (0.89, 0.042228165302860006, 0.254687844518532),
    (0.90, 0.04542119807150263, 0.2480842411779343),
    (0.91, 0.04888601735264928, 0.24123680380179505),
    (0.92, 0.05266677984293328, 0.23410107386271845),
    (0.93, 0.05682194002225034, 0.22661829608964376),
    (0.94, 0.06143173695676035, 0.2187079319185452),
    (0.95, 0.06661162923820178, 0.21025422478526803),
)


def coexistence_densities(T_over_Tc):
    """(rho_g, rho_l) at T/T_c, linearly interpolated in COEXISTENCE_CS (0.60..0.95)."""
    t = np.array([r[0] for r in COEXISTENCE_CS])
    if not (t[0] - 1e-12 <= T_over_Tc <= t[-1] + 1e-12):
        raise ValueError(f"T/T_c = {T_over_Tc} outside the table")
    g = float(np.interp(T_over_Tc, t, [r[1] for r in COEXISTENCE_CS]))
    l = float(np.interp(T_over_Tc, t, [r[2] for r in COEXISTENCE_CS]))
    return g, l

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """One SplitMix64 output for each 64-bit state in x (vectorised)."""
    with np.errstate(over="ignore"):
        z = (np.asarray(x, dtype=np.uint64) + np.uint64(0x9E3779B97F4A7C15)) & _M64
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _M64
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _M64
        return z ^ (z >> np.uint64(31))


def uniform01(seed: int, index: np.ndarray) -> np.ndarray:
    """Counter-based U[0, 1) doubles: SplitMix64(SplitMix64(seed) ^ index) >> 11."""
    key = splitmix64(np.array([seed], dtype=np.uint64))[0]
    z = splitmix64(np.asarray(index, dtype=np.uint64) ^ key)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def site_noise(seed: int, nx: int, ny: int, amplitude: float) -> np.ndarray:
    """Noise U[-amplitude, amplitude] on an ny x nx lattice, site s = y*nx + x."""
    idx = np.arange(nx * ny, dtype=np.uint64)
    return (amplitude * (2.0 * uniform01(seed, idx) - 1.0)).reshape(ny, nx)


def slab_fields(nx, ny, T_over_Tc=0.85, width=32, rho_l=RHO_LIQUID, rho_g=RHO_GAS,
                noise=1e-3, seed=1, Tc=CS_TC):
    """Flat liquid slab x in [nx/2 - width/2, nx/2 + width/2) plus noise; uniform T."""
    x = np.arange(nx)
    liquid = (x >= nx // 2 - width // 2) & (x < nx // 2 + width // 2)
    rho = np.where(liquid[None, :], rho_l, rho_g) * np.ones((ny, 1))
    if noise:
        rho = rho + site_noise(seed, nx, ny, noise)
    T = np.full((ny, nx), T_over_Tc * Tc)
    return np.ascontiguousarray(rho), T


def droplet_fields(nx, ny, radius, T_lo=0.80, T_hi=0.90, rho_l=RHO_LIQUID,
                   rho_g=RHO_GAS, Tc=CS_TC, noise=0.0, seed=2):
    """Sharp droplet centred at (nx/2, ny/2); T linear in x from T_lo to T_hi (x T_c).

    The linear profile is taken literally on the periodic lattice, so T jumps
    at the x seam.
    """
    y, x = np.mgrid[0:ny, 0:nx]
    r2 = (x - nx / 2 + 0.5) ** 2 + (y - ny / 2 + 0.5) ** 2
    rho = np.where(r2 < radius * radius, rho_l, rho_g).astype(np.float64)
    if noise:
        rho = rho + site_noise(seed, nx, ny, noise)
    T = Tc * (T_lo + (T_hi - T_lo) * x / (nx - 1))
    return np.ascontiguousarray(rho), np.ascontiguousarray(T.astype(np.float64))


def spinodal_fields(nx, ny, T_over_Tc=0.75, rho_mean=0.12, noise=0.01, seed=3, Tc=CS_TC):
    """Uniform density rho_mean plus seeded noise, uniform T: spinodal decomposition."""
    rho = rho_mean + site_noise(seed, nx, ny, noise)
    T = np.full((ny, nx), T_over_Tc * Tc)
    return np.ascontiguousarray(rho), T


def uniform_fields(nx, ny, rho, T):
    return np.full((ny, nx), float(rho)), np.full((ny, nx), float(T))


def sinusoid_fields(nx, ny, rho0, T0, eps, mode=1, axis=0):
    """rho = rho0 (1 + eps sin(k x)) with k = 2 pi mode / nx (axis 0 = x); uniform T."""
    if axis == 0:
        k = 2.0 * np.pi * mode / nx
        prof = np.sin(k * np.arange(nx))[None, :] * np.ones((ny, 1))
    else:
        k = 2.0 * np.pi * mode / ny
        prof = np.sin(k * np.arange(ny))[:, None] * np.ones((1, nx))
    rho = rho0 * (1.0 + eps * prof)
    return np.ascontiguousarray(rho), np.full((ny, nx), float(T0))


@dataclasses.dataclass
class Domain:
    """One domain of the batched parameter sweep."""

    L: int
    T_over_Tc: float
    G: float
    tau_f: float
    tau_g: float
    kind: str           # "droplet" or "slab"
    size: float         # droplet radius or slab width
    rho: np.ndarray
    T: np.ndarray


def batched_sweep(n_domains=256, L_min=64, L_max=512, seed=4, tau_g=0.8, Tc=CS_TC,
                  fixed_L=None, L_multiple=1, densities="coexistence"):
    """Parameter sweep of independent periodic square domains.

    Per domain d (stream index 16 d + k of the counter-based generator):
    side L ~ U{L_min..L_max} (rounded down to a multiple of L_multiple; 1, the
    default, keeps the drawn side),
    T/T_c ~ U[0.6, 0.95], G ~ U[-1.2, -0.8],
    tau_f ~ U[0.6, 1.2], tau_g fixed; droplet (radius U[L/8, L/4]) or slab
    (width U[L/4, L/2]) from a fair coin.  densities="coexistence" starts the
    liquid and the vapour at the EOS coexistence densities of the domain's
    T/T_c (COEXISTENCE_CS); "fixed" at RHO_LIQUID / RHO_GAS.
    """
    out = []
    for d in range(n_domains):
        u = uniform01(seed, np.arange(16 * d, 16 * d + 8, dtype=np.uint64))
        L = int(fixed_L) if fixed_L else int(L_min + min(int(u[0] * (L_max - L_min + 1)),
                                                         L_max - L_min))
        L -= L % L_multiple
        T_over = 0.6 + 0.35 * u[1]
        G = -1.2 + 0.4 * u[2]
        tau_f = 0.6 + 0.6 * u[3]
        rg, rl = coexistence_densities(T_over) if densities == "coexistence" else (RHO_GAS, RHO_LIQUID)
        if u[4] < 0.5:
            kind = "droplet"
            size = L / 8 + (L / 4 - L / 8) * u[5]
            rho, _ = droplet_fields(L, L, size, rho_l=rl, rho_g=rg)
        else:
            kind = "slab"
            size = L / 4 + (L / 2 - L / 4) * u[5]
            w = max(2, 2 * int(size / 2))
            rho, _ = slab_fields(L, L, width=w, rho_l=rl, rho_g=rg, noise=0.0)
        T = np.full((L, L), T_over * Tc)
        out.append(Domain(L, float(T_over), float(G), float(tau_f), float(tau_g), kind,
                          float(size), rho, T))
    return out


# ------------------------------------------------------- warm-start network
#: Normalisation of the network's input planes and outputs:
#: input (T/T_c - t_mid)/t_scale, (G - g_mid)/g_scale, 2 mask - 1;
#: output (deviations from the case's initial fields rho0, T0):
#: rho = rho0 + rho_dev_scale y0, T = T0 (1 + t_dev_scale y1).
UNET_NORM = dict(t_mid=0.775, t_scale=0.1, g_mid=-1.0, g_scale=0.2, rho_dev_scale=0.1,
                 t_dev_scale=0.001)


def normal01(seed: int, index: np.ndarray) -> np.ndarray:
    """Counter-based standard normals (Box-Muller on uniform01(seed, 2i), (2i+1))."""
    i = np.asarray(index, dtype=np.uint64)
    u1 = uniform01(seed, np.uint64(2) * i)
    u2 = uniform01(seed, np.uint64(2) * i + np.uint64(1))
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)


def unet_init_params(layers, seed=11) -> np.ndarray:
    """He-normal initial parameters (float32 values) for a layer list of
    (name, cin_stored, cout, ksize, cin_real): W[cout, k, k, cin_stored] with
    std sqrt(2 / (k^2 cin_real)) for 3x3 layers and sqrt(1 / cin_real) for the
    1x1 head, zero for input channels >= cin_real (padding); biases zero.
    Flat order: W then b, layer by layer."""
    out, base = [], 0
    for _, ci, co, k, ci_real in layers:
        n = co * k * k * ci
        std = np.sqrt((2.0 if k == 3 else 1.0) / (k * k * ci_real))
        W = (normal01(seed, np.arange(base, base + n, dtype=np.uint64)) * std).reshape(co, k, k, ci)
        W[..., ci_real:] = 0.0
        out += [W.reshape(-1), np.zeros(co)]
        base += n
    return np.concatenate(out).astype(np.float32)


def unet_input_planes(T_over_Tc, G, mask) -> np.ndarray:
    """Network input [N, H, W, 3] float32 from per-case T/T_c [N], G [N] and
    initial liquid masks [N, H, W] (1 inside the droplet/slab)."""
    m = np.asarray(mask, dtype=np.float64)
    n = m.shape[0]
    t = ((np.asarray(T_over_Tc, dtype=np.float64) - UNET_NORM["t_mid"]) / UNET_NORM["t_scale"]).reshape(n, 1, 1)
    g = ((np.asarray(G, dtype=np.float64) - UNET_NORM["g_mid"]) / UNET_NORM["g_scale"]).reshape(n, 1, 1)
    return np.stack([np.broadcast_to(t, m.shape), np.broadcast_to(g, m.shape), 2.0 * m - 1.0],
                    axis=3).astype(np.float32)


def unet_target_planes(rho, T, rho0, T0) -> np.ndarray:
    """Normalised training targets [N, H, W, 2] float32 from steady rho, T fields
    and the cases' initial fields rho0 [N, H, W] and temperatures T0 (scalars
    [N] or fields)."""
    r = (np.asarray(rho, dtype=np.float64) - np.asarray(rho0, dtype=np.float64)) / UNET_NORM["rho_dev_scale"]
    T = np.asarray(T, dtype=np.float64)
    T0 = np.asarray(T0, dtype=np.float64)
    if T0.ndim == 1:
        T0 = T0.reshape(-1, 1, 1)
    t = (T / T0 - 1.0) / UNET_NORM["t_dev_scale"]
    return np.stack([r, t], axis=-1).astype(np.float32)


def warm_start_cases(n, L=256, seed=5):
    """n sweep cases at a fixed L x L (the batched sweep's parameter
    distributions); returns the domains and their initial liquid masks."""
    doms = batched_sweep(n_domains=n, seed=seed, fixed_L=L)
    masks = np.stack([(d.rho > 0.5 * (d.rho.max() + d.rho.min())).astype(np.float32) for d in doms])
    return doms, masks
