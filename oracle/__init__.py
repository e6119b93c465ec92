"""Plain FP64 CPU oracle of the thermal pseudopotential D2Q9 LB step.

TEST INFRASTRUCTURE ONLY.  The oracle is the slow, obviously correct
reference written from the equations of Li & Luo (arXiv:1405.2232):
Eq. (1) with the forcing term of Ref. [21], Eqs. (2)/(4) for the force,
the pseudopotential of Sec. II A, Eq. (7) and Eqs. (24)-(25) for the
temperature distribution.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
it.  It shares no code with the CUDA library and never imports it.

All arrays are float64 numpy arrays.  Populations use the layout
``f[i, y, x]`` (nine planes, row-major), holding the PRE-collision values at
the current time.

Parity status of each function (what pins it, see tests/test_oracle_pins.py):
  feq, forcing_term, correction_term  -- exact moment identities
  p_eos / critical_point             -- vdW closed form, published CS critical
                                        point, hard-sphere virial coefficients
  force (Eq. 2/4)                    -- closed form on a sinusoid, Taylor limit
  step                               -- conservation, uniform state,
                                        translation, G and c_v invariance,
                                        Chapman-Enskog drift rate (Eq. 23)
                                        and steady states (Eq. 23 / A11),
                                        brute-force per-site recomputation
  fd_rhs, fd_rk2, step_fd (Eqs. 26-27) -- closed-form eigenvalues of the
                                        isotropic gradient and Laplacian on
                                        Fourier modes, RK2 amplification
                                        factors, uniform-state invariance
  unet (warm-start network)          -- see oracle/unet.py
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lb_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liblboracle.so")
_lock = threading.Lock()
_lib = None

EOS_CS, EOS_VDW, EOS_IDEAL = 0, 1, 2
THERMAL_EQ7, THERMAL_EQ24 = 0, 1

OK, ERR_ARG, ERR_NONFINITE, ERR_PSI_DOMAIN = 0, 1, 4, 5


class OracleParams(ctypes.Structure):
    """Mirror of the oracle's own ``or_params`` struct."""

    _fields_ = [
        ("nx", ctypes.c_int32),
        ("ny", ctypes.c_int32),
        ("tau_f", ctypes.c_double),
        ("tau_g", ctypes.c_double),
        ("G", ctypes.c_double),
        ("beta", ctypes.c_double),
        ("eos", ctypes.c_int32),
        ("a", ctypes.c_double),
        ("b", ctypes.c_double),
        ("R", ctypes.c_double),
        ("cv", ctypes.c_double),
        ("thermal", ctypes.c_int32),
        ("psi_uses_local_T", ctypes.c_int32),
        ("T_psi", ctypes.c_double),
    ]


class OracleChannel(ctypes.Structure):
    """Inlet and plate conditions of the channel (Sec. III A)."""
    _fields_ = [("T_in", ctypes.c_double), ("T_w", ctypes.c_double), ("U_in", ctypes.c_double),
                ("adiabatic_bottom", ctypes.c_int32)]


class OracleCavity(ctypes.Structure):
    """Side-wall temperatures and gravity of the cavity (Sec. III B)."""
    _fields_ = [("T_hot", ctypes.c_double), ("T_cold", ctypes.c_double), ("g_grav", ctypes.c_double)]



def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP contraction off, OpenMP on)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
           "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def build_variant(source_text: str, tag: str) -> str:
    """Compile a modified copy of the oracle source (used by the mutation tests,
    which plant a mistake in the oracle and check that a pin catches it)."""
    os.makedirs(_BUILD, exist_ok=True)
    src = os.path.join(_BUILD, f"variant_{tag}.c")
    lib = os.path.join(_BUILD, f"libvariant_{tag}.so")
    with open(src, "w") as fh:
        fh.write(source_text)
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                    "-fPIC", "-shared", src, "-o", lib, "-lm"], check=True)
    return lib


def source_text() -> str:
    with open(_SRC) as fh:
        return fh.read()


class using:
    """Context manager: route every oracle call to another build of the source."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib
        self._saved = _lib
        _lib = _bind(ctypes.CDLL(self.path))
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self._saved
        return False


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        _lib = _bind(ctypes.CDLL(build()))
        return _lib


def _bind(lib):
    """Declare the C signatures on a loaded oracle library."""
    dp = ctypes.POINTER(ctypes.c_double)
    P = ctypes.POINTER(OracleParams)
    lib.or_p_eos.argtypes = [P, ctypes.c_double, ctypes.c_double]
    lib.or_p_eos.restype = ctypes.c_double
    lib.or_psi_sq.argtypes = [P, ctypes.c_double, ctypes.c_double]
    lib.or_psi_sq.restype = ctypes.c_double
    lib.or_feq.argtypes = [ctypes.c_double] * 3 + [dp]
    lib.or_forcing_term.argtypes = [ctypes.c_double] * 5 + [dp]
    lib.or_correction_term.argtypes = [ctypes.c_double] * 5 + [dp]
    lib.or_step.argtypes = [P, dp, dp, dp, dp, ctypes.c_int]
    lib.or_step.restype = ctypes.c_int
    lib.or_moments.argtypes = [P, dp, dp, dp, dp, dp, dp, dp, dp]
    lib.or_moments.restype = ctypes.c_int
    lib.or_init_equilibrium.argtypes = [P, dp, dp, dp, dp]
    lib.or_init_equilibrium.restype = ctypes.c_int
    lib.or_init_balanced.argtypes = [P, dp, dp, dp, dp]
    lib.or_init_balanced.restype = ctypes.c_int
    lib.or_step_sites.argtypes = [P, dp, dp, ctypes.c_int64,
                                  ctypes.POINTER(ctypes.c_int64), dp, dp]
    lib.or_step_sites.restype = ctypes.c_int
    lib.or_totals.argtypes = [P, dp, dp, dp]
    lib.or_totals.restype = ctypes.c_int
    lib.or_residual.argtypes = [ctypes.c_int64, dp, dp, dp, dp, ctypes.c_int64]
    lib.or_residual.restype = ctypes.c_double
    lib.or_critical_point.argtypes = [P, dp, dp]
    lib.or_critical_point.restype = ctypes.c_int
    lib.or_num_threads_available.restype = ctypes.c_int
    lib.or_fd_rhs.argtypes = [P, dp, dp, dp, dp, dp]
    lib.or_fd_rhs.restype = None
    lib.or_fd_rk2.argtypes = [P, dp, dp, dp, dp, ctypes.c_int, dp]
    lib.or_fd_rk2.restype = ctypes.c_int
    lib.or_step_fd.argtypes = [P, dp, dp, dp, dp, ctypes.c_int, dp, dp, dp, ctypes.c_int]
    lib.or_step_fd.restype = ctypes.c_int
    Cv = ctypes.POINTER(OracleCavity)
    lib.or_step_cavity.argtypes = [P, Cv, dp, dp, dp, dp, ctypes.c_int]
    lib.or_step_cavity.restype = ctypes.c_int
    lib.or_nusselt_hot.argtypes = [P, Cv, dp]
    lib.or_nusselt_hot.restype = ctypes.c_double
    lib.or_nusselt_hot_flux.argtypes = [P, Cv, dp, dp]
    lib.or_nusselt_hot_flux.restype = ctypes.c_double
    lib.or_step_fd_cavity.argtypes = [P, Cv, dp, dp, dp, dp, ctypes.c_int, dp, dp, dp, ctypes.c_int]
    lib.or_step_fd_cavity.restype = ctypes.c_int
    lib.or_nusselt_hot_wall.argtypes = [P, Cv, dp, dp]
    lib.or_nusselt_hot_wall.restype = ctypes.c_double
    Ch = ctypes.POINTER(OracleChannel)
    lib.or_step_channel.argtypes = [P, Ch, dp, dp, dp, dp, ctypes.c_int]
    lib.or_step_channel.restype = ctypes.c_int
    lib.or_channel_nusselt.argtypes = [P, Ch, dp, dp, dp, dp, ctypes.c_int]
    lib.or_channel_nusselt.restype = ctypes.c_double
    lib.or_channel_nusselt_grad.argtypes = [P, Ch, dp, dp, dp, ctypes.c_int]
    lib.or_channel_nusselt_grad.restype = ctypes.c_double
    lib.or_step_fd_channel.argtypes = [P, Ch, dp, dp, dp, dp, ctypes.c_int, dp, dp, dp, ctypes.c_int]
    lib.or_step_fd_channel.restype = ctypes.c_int
    lib.or_channel_nusselt_wall.argtypes = [P, Ch, dp, dp, dp, ctypes.c_int]
    lib.or_channel_nusselt_wall.restype = ctypes.c_double
    return lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def params(nx, ny, tau_f=1.0, tau_g=0.8, G=-1.0, beta=1.0, eos=EOS_CS, a=1.0, b=4.0,
           R=1.0, cv=1.0, thermal=THERMAL_EQ24, psi_uses_local_T=1, T_psi=0.0):
    """Build the oracle's parameter struct (names follow the paper)."""
    return OracleParams(int(nx), int(ny), float(tau_f), float(tau_g), float(G),
                        float(beta), int(eos), float(a), float(b), float(R),
                        float(cv), int(thermal), int(psi_uses_local_T), float(T_psi))


def p_eos(P, rho, T):
    return _load().or_p_eos(ctypes.byref(P), float(rho), float(T))


def psi_sq(P, rho, T):
    return _load().or_psi_sq(ctypes.byref(P), float(rho), float(T))


def feq(rho, ux, uy):
    out = np.zeros(9)
    _load().or_feq(float(rho), float(ux), float(uy), _ptr(out))
    return out


def forcing_term(tau_f, ux, uy, Fx, Fy):
    out = np.zeros(9)
    _load().or_forcing_term(float(tau_f), float(ux), float(uy), float(Fx), float(Fy),
                            _ptr(out))
    return out


def correction_term(tau_g, cv, T, Fx, Fy):
    out = np.zeros(9)
    _load().or_correction_term(float(tau_g), float(cv), float(T), float(Fx), float(Fy),
                               _ptr(out))
    return out


def init_equilibrium(P, rho0, T0):
    """f = f^eq(rho0, 0), g = c_v T0 f^eq(rho0, 0): arrays [9, ny, nx]."""
    rho0 = np.ascontiguousarray(rho0, dtype=np.float64)
    T0 = np.ascontiguousarray(T0, dtype=np.float64)
    assert rho0.shape == (P.ny, P.nx) and T0.shape == (P.ny, P.nx)
    f = np.zeros((9, P.ny, P.nx))
    g = np.zeros((9, P.ny, P.nx))
    rc = _load().or_init_equilibrium(ctypes.byref(P), _ptr(rho0), _ptr(T0), _ptr(f), _ptr(g))
    if rc:
        raise ValueError(f"or_init_equilibrium failed: {rc}")
    return f, g


def init_balanced(P, rho0, T0):
    """State at rest under the force: f = f^eq(rho0, v), g = c_v T0 f^eq(rho0, v)
    with v = -F/(2 rho0), F the Eq. (4) force of psi(rho0, T0); returns
    (f, g, status), status ERR_PSI_DOMAIN where psi is undefined."""
    rho0 = np.ascontiguousarray(rho0, dtype=np.float64)
    T0 = np.ascontiguousarray(T0, dtype=np.float64)
    assert rho0.shape == (P.ny, P.nx) and T0.shape == (P.ny, P.nx)
    f = np.zeros((9, P.ny, P.nx))
    g = np.zeros((9, P.ny, P.nx))
    rc = _load().or_init_balanced(ctypes.byref(P), _ptr(rho0), _ptr(T0), _ptr(f), _ptr(g))
    if rc == ERR_ARG:
        raise ValueError("or_init_balanced: invalid parameters")
    return f, g, rc


def step(P, f, g, n=1, threads=1, check=True):
    """Advance the pre-collision state (f, g) by n steps; returns (f, g, status)."""
    f = np.ascontiguousarray(f, dtype=np.float64).copy()
    g = np.ascontiguousarray(g, dtype=np.float64).copy()
    fn = np.empty_like(f)
    gn = np.empty_like(g)
    lib = _load()
    worst = OK
    for _ in range(int(n)):
        rc = lib.or_step(ctypes.byref(P), _ptr(f), _ptr(g), _ptr(fn), _ptr(gn), int(threads))
        if rc == ERR_ARG:
            raise ValueError("or_step: invalid parameters")
        worst = max(worst, rc)
        f, fn = fn, f
        g, gn = gn, g
    if check and worst:
        raise FloatingPointError(f"oracle step reported status {worst}")
    return f, g, worst


def moments(P, f, g):
    """(rho, ux, uy, T, Fx, Fy) of the pre-collision state, each [ny, nx]."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    outs = [np.zeros((P.ny, P.nx)) for _ in range(6)]
    rc = _load().or_moments(ctypes.byref(P), _ptr(f), _ptr(g), *[_ptr(o) for o in outs])
    if rc == ERR_ARG:
        raise ValueError("or_moments: invalid parameters")
    return tuple(outs)


def step_sites(P, f, g, sites):
    """State at t+1 at the given flat site indices; returns (f, g) as [n, 9]."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    sites = np.ascontiguousarray(sites, dtype=np.int64)
    of = np.zeros((len(sites), 9))
    og = np.zeros((len(sites), 9))
    rc = _load().or_step_sites(ctypes.byref(P), _ptr(f), _ptr(g), len(sites),
                               sites.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                               _ptr(of), _ptr(og))
    if rc == ERR_ARG:
        raise ValueError("or_step_sites: invalid arguments")
    return of, og


def _field(a, P):
    a = np.ascontiguousarray(a, dtype=np.float64)
    assert a.shape == (P.ny, P.nx)
    return a


def fd_rhs(P, T, rho, ux, uy):
    """K(T) of Eq. (26) at every site ([ny, nx])."""
    T, rho, ux, uy = (_field(a, P) for a in (T, rho, ux, uy))
    K = np.zeros((P.ny, P.nx))
    _load().or_fd_rhs(ctypes.byref(P), _ptr(T), _ptr(rho), _ptr(ux), _ptr(uy), _ptr(K))
    return K


def fd_rk2(P, T, rho, ux, uy, printed=False):
    """One Eq. (27) update of T with rho, u fixed (printed: a = 1/2, else Heun)."""
    T, rho, ux, uy = (_field(a, P) for a in (T, rho, ux, uy))
    Tn = np.zeros((P.ny, P.nx))
    rc = _load().or_fd_rk2(ctypes.byref(P), _ptr(T), _ptr(rho), _ptr(ux), _ptr(uy), int(bool(printed)), _ptr(Tn))
    if rc == ERR_ARG:
        raise ValueError("or_fd_rk2 failed")
    return Tn


def step_fd(P, f, T, n=1, printed=False, threads=1, check=True):
    """n steps of the hybrid scheme (f by Eq. (1), T by Eqs. (26)-(27)).
    Returns (f, T, status, (rho, ux, uy) of the last step's time level)."""
    f = np.ascontiguousarray(f, dtype=np.float64).copy()
    T = _field(T, P).copy()
    fn, Tn = np.empty_like(f), np.empty_like(T)
    rho, ux, uy = (np.zeros((P.ny, P.nx)) for _ in range(3))
    worst = OK
    for _ in range(int(n)):
        rc = _load().or_step_fd(ctypes.byref(P), _ptr(f), _ptr(T), _ptr(fn), _ptr(Tn), int(bool(printed)),
                                _ptr(rho), _ptr(ux), _ptr(uy), int(threads))
        if rc == ERR_ARG:
            raise ValueError("or_step_fd: invalid parameters")
        worst = max(worst, rc)
        f, fn = fn, f
        T, Tn = Tn, T
    if check and worst:
        raise FloatingPointError(f"oracle FD step reported status {worst}")
    return f, T, worst, (rho, ux, uy)


def totals(P, f, g):
    """[mass, energy, px, py] with compensated summation."""
    out = np.zeros(4)
    f = np.ascontiguousarray(f, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    _load().or_totals(ctypes.byref(P), _ptr(f), _ptr(g), _ptr(out))
    return out


def residual(rho0, T0, rho1, T1, K):
    """max over {rho, T} of ||phi1 - phi0||_2 / (K ||phi1||_2)."""
    arrs = [np.ascontiguousarray(a, dtype=np.float64).ravel() for a in (rho0, T0, rho1, T1)]
    return _load().or_residual(arrs[0].size, *[_ptr(a) for a in arrs], int(K))


def critical_point(P):
    """(T_c, rho_c) of the EOS in P, from dp/drho = d2p/drho2 = 0."""
    Tc = ctypes.c_double()
    rc_ = ctypes.c_double()
    rc = _load().or_critical_point(ctypes.byref(P), ctypes.byref(Tc), ctypes.byref(rc_))
    if rc:
        raise ValueError("no critical point for this EOS")
    return Tc.value, rc_.value


def threads_available():
    return _load().or_num_threads_available()


# ------------------------------------------------------------------ cavity
def cavity(T_hot=1.03, T_cold=0.97, g_grav=0.0):
    return OracleCavity(float(T_hot), float(T_cold), float(g_grav))


def cavity_setup(Ra, L, thermal=THERMAL_EQ24, T_hot=1.03, T_cold=0.97, mu=0.1, Pr=0.71, rho0=1.0):
    """Parameters of the natural-convection cavity of Sec. III B on an L x L
    lattice: ideal EOS with R = 1/3 (c = sqrt(3 R T_c) = 1 at T_c = 1), the
    pseudopotential in the beta = 0 form of Eq. (4), tau_f from mu = rho0 cs^2
    (tau_f - 1/2), tau_g from Pr = nu / chi with chi = cs^2 (tau_g - 1/2), and g
    from Eq. (28) with beta_T = 1/T_c.  Returns (P, Cv)."""
    Tc = 0.5 * (T_hot + T_cold)
    R = 1.0 / (3.0 * Tc)
    nu = mu / rho0
    tau_f = 0.5 + 3.0 * nu
    tau_g = 0.5 + 3.0 * nu / Pr
    g = Ra * mu * mu / ((1.0 / Tc) * rho0 * rho0 * (T_hot - T_cold) * L ** 3 * Pr)
    P = params(L, L, tau_f=tau_f, tau_g=tau_g, G=-1.0, beta=0.0, eos=EOS_IDEAL, R=R, cv=1.0,
               thermal=thermal, psi_uses_local_T=1)
    return P, cavity(T_hot, T_cold, g)


def step_cavity(P, Cv, f, g, n=1, threads=1, check=True):
    """Advance the cavity state (f, g) by n steps; returns (f, g, status)."""
    f = np.ascontiguousarray(f, dtype=np.float64).copy()
    g = np.ascontiguousarray(g, dtype=np.float64).copy()
    fn = np.empty_like(f)
    gn = np.empty_like(g)
    lib = _load()
    worst = OK
    for _ in range(int(n)):
        rc = lib.or_step_cavity(ctypes.byref(P), ctypes.byref(Cv), _ptr(f), _ptr(g), _ptr(fn), _ptr(gn),
                                int(threads))
        if rc == ERR_ARG:
            raise ValueError("or_step_cavity: invalid parameters")
        worst = max(worst, rc)
        f, fn = fn, f
        g, gn = gn, g
    if check and worst:
        raise FloatingPointError(f"oracle cavity step reported status {worst}")
    return f, g, worst


def nusselt_hot(P, Cv, T):
    """Average Nusselt number at the hot wall from the temperature gradient
    (as Table II), T [ny, nx]."""
    T = _field(T, P)
    return _load().or_nusselt_hot(ctypes.byref(P), ctypes.byref(Cv), _ptr(T))


def nusselt_hot_flux(P, Cv, f, g):
    """Average Nusselt number at the hot wall from the energy flux through the
    wall links of the pre-collision state."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    return _load().or_nusselt_hot_flux(ctypes.byref(P), ctypes.byref(Cv), _ptr(f), _ptr(g))


def step_fd_cavity(P, Cv, f, T, n=1, printed=False, threads=1, check=True):
    """n steps of the hybrid scheme in the cavity; returns (f, T, status, (rho, ux, uy))."""
    f = np.ascontiguousarray(f, dtype=np.float64).copy()
    T = _field(T, P).copy()
    fn, Tn = np.empty_like(f), np.empty_like(T)
    rho, ux, uy = (np.zeros((P.ny, P.nx)) for _ in range(3))
    worst = OK
    for _ in range(int(n)):
        rc = _load().or_step_fd_cavity(ctypes.byref(P), ctypes.byref(Cv), _ptr(f), _ptr(T), _ptr(fn), _ptr(Tn),
                                       int(bool(printed)), _ptr(rho), _ptr(ux), _ptr(uy), int(threads))
        if rc == ERR_ARG:
            raise ValueError("or_step_fd_cavity: invalid parameters")
        worst = max(worst, rc)
        f, fn = fn, f
        T, Tn = Tn, T
    if check and worst:
        raise FloatingPointError(f"oracle FD cavity step reported status {worst}")
    return f, T, worst, (rho, ux, uy)


def nusselt_hot_wall(P, Cv, T, rho=None):
    """Nusselt number at the hot wall from the central difference across it
    (T at the wall imposed through the reflected ghost, the FD treatment);
    with rho, the conductive flux lambda(rho) dT/dx normalised by lambda0."""
    T = _field(T, P)
    if rho is None:
        return _load().or_nusselt_hot_wall(ctypes.byref(P), ctypes.byref(Cv), _ptr(T), None)
    rho = _field(rho, P)
    return _load().or_nusselt_hot_wall(ctypes.byref(P), ctypes.byref(Cv), _ptr(T), _ptr(rho))


# ------------------------------------------------------------------ channel
def channel_setup(nx, ny, case="A", thermal=THERMAL_EQ24, T_in=1.03, T_w=0.97, U_in=0.05, mu=0.1, Pr=0.71,
                  rho0=1.0):
    """Parameters of the plate-channel test of Sec. III A on an nx x ny
    lattice: ideal EOS with R = 1/3 (c = sqrt(3 R T_c) = 1 at T_c = (T_in +
    T_w)/2 = 1), the pseudopotential in the beta = 0 form of Eq. (4), tau_f
    from mu = rho0 cs^2 (tau_f - 1/2), tau_g from Pr.  Case A: both plates at
    T_w; Case B: the lower plate adiabatic.  Returns (P, Ch)."""
    Tc = 0.5 * (T_in + T_w)
    nu = mu / rho0
    P = params(nx, ny, tau_f=0.5 + 3.0 * nu, tau_g=0.5 + 3.0 * nu / Pr, G=-1.0, beta=0.0, eos=EOS_IDEAL,
               R=1.0 / (3.0 * Tc), cv=1.0, thermal=thermal, psi_uses_local_T=1)
    return P, OracleChannel(float(T_in), float(T_w), float(U_in), 1 if case == "B" else 0)


def step_channel(P, Ch, f, g, n=1, threads=1, check=True):
    """Advance the channel state (f, g) by n steps; returns (f, g, status)."""
    f = np.ascontiguousarray(f, dtype=np.float64).copy()
    g = np.ascontiguousarray(g, dtype=np.float64).copy()
    fn = np.empty_like(f)
    gn = np.empty_like(g)
    lib = _load()
    worst = OK
    for _ in range(int(n)):
        rc = lib.or_step_channel(ctypes.byref(P), ctypes.byref(Ch), _ptr(f), _ptr(g), _ptr(fn), _ptr(gn),
                                 int(threads))
        if rc == ERR_ARG:
            raise ValueError("or_step_channel: invalid parameters")
        worst = max(worst, rc)
        f, fn = fn, f
        g, gn = gn, g
    if check and worst:
        raise FloatingPointError(f"oracle channel step reported status {worst}")
    return f, g, worst


def channel_nusselt(P, Ch, g, rho, ux, T, x):
    """Local Nusselt number at column x from the upper plate's heat flux."""
    g = np.ascontiguousarray(g, dtype=np.float64)
    rho, ux, T = (_field(a, P) for a in (rho, ux, T))
    return _load().or_channel_nusselt(ctypes.byref(P), ctypes.byref(Ch), _ptr(g), _ptr(rho), _ptr(ux), _ptr(T),
                                      int(x))


def channel_nusselt_grad(P, Ch, rho, ux, T, x):
    """Local Nusselt number at column x from the temperature gradient at the upper plate."""
    rho, ux, T = (_field(a, P) for a in (rho, ux, T))
    return _load().or_channel_nusselt_grad(ctypes.byref(P), ctypes.byref(Ch), _ptr(rho), _ptr(ux), _ptr(T), int(x))


def step_fd_channel(P, Ch, f, T, n=1, printed=False, threads=1, check=True):
    """n steps of the hybrid scheme in the channel; returns (f, T, status, (rho, ux, uy))."""
    f = np.ascontiguousarray(f, dtype=np.float64).copy()
    T = _field(T, P).copy()
    fn, Tn = np.empty_like(f), np.empty_like(T)
    rho, ux, uy = (np.zeros((P.ny, P.nx)) for _ in range(3))
    worst = OK
    for _ in range(int(n)):
        rc = _load().or_step_fd_channel(ctypes.byref(P), ctypes.byref(Ch), _ptr(f), _ptr(T), _ptr(fn), _ptr(Tn),
                                        int(bool(printed)), _ptr(rho), _ptr(ux), _ptr(uy), int(threads))
        if rc == ERR_ARG:
            raise ValueError("or_step_fd_channel: invalid parameters")
        worst = max(worst, rc)
        f, fn = fn, f
        T, Tn = Tn, T
    if check and worst:
        raise FloatingPointError(f"oracle FD channel step reported status {worst}")
    return f, T, worst, (rho, ux, uy)


def channel_nusselt_wall(P, Ch, rho, ux, T, x):
    """Local Nusselt number at column x, plate gradient across the plate (FD)."""
    rho, ux, T = (_field(a, P) for a in (rho, ux, T))
    return _load().or_channel_nusselt_wall(ctypes.byref(P), ctypes.byref(Ch), _ptr(rho), _ptr(ux), _ptr(T), int(x))
