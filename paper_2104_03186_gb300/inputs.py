"""Seeded synthetic LQT workloads.

This module only draws inputs: dynamics (F_k, c_k, L_k), costs (H_k, r_k, X_k,
U_k), terminal terms (H_T, r_T, X_T) and the initial state x_0 of the LQT
problem of Sec. II-B (eq. LQT_problem).  It holds none of the solver's
arithmetic, so the CUDA path and the FP64 oracle can both be fed from it.

Per-step arrays carry a leading time axis of length T, or of length 1 for a
matrix that is the same at every step (a step stride of 0 at the C ABI).
All arrays are float64 and C-contiguous; ``LQTProblem.astype`` casts them.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

STEP_FIELDS = ("F", "c", "L", "U", "H", "r", "X")


@dataclasses.dataclass
class LQTProblem:
    F: np.ndarray            # (1|T, n, n)
    c: Optional[np.ndarray]  # (1|T, n) or None (= 0)
    L: np.ndarray            # (1|T, n, m)
    U: np.ndarray            # (1|T, m, m)
    H: np.ndarray            # (1|T, p, n)
    r: Optional[np.ndarray]  # (1|T, p) or None (= 0)
    X: np.ndarray            # (1|T, p, p)
    HT: np.ndarray           # (pT, n)
    rT: Optional[np.ndarray] # (pT,) or None (= 0)
    XT: np.ndarray           # (pT, pT)
    x0: np.ndarray           # (n,)
    T: int

    @property
    def n(self) -> int:
        return int(self.F.shape[-1])

    @property
    def m(self) -> int:
        return int(self.L.shape[-1])

    @property
    def p(self) -> int:
        return int(self.H.shape[-2])

    @property
    def pT(self) -> int:
        return int(self.HT.shape[0])

    def time_invariant(self, name: str) -> bool:
        a = getattr(self, name)
        return a is None or a.shape[0] == 1

    def astype(self, dtype) -> "LQTProblem":
        def cast(a):
            return None if a is None else np.ascontiguousarray(a, dtype=dtype)

        return dataclasses.replace(
            self, **{f.name: cast(getattr(self, f.name))
                     for f in dataclasses.fields(self) if f.name != "T"})

    def rounded_to(self, dtype) -> "LQTProblem":
        """Round every input to ``dtype`` and back to float64, so that a
        lower-precision solver and a float64 reference see identical values."""
        return self.astype(dtype).astype(np.float64)

    def check(self) -> None:
        n, m, p, T = self.n, self.m, self.p, self.T
        shapes = {"F": (n, n), "c": (n,), "L": (n, m), "U": (m, m),
                  "H": (p, n), "r": (p,), "X": (p, p)}
        for name, tail in shapes.items():
            a = getattr(self, name)
            if a is None:
                continue
            assert a.shape[1:] == tail, (name, a.shape, tail)
            assert a.shape[0] in (1, T), (name, a.shape, T)
        assert self.HT.shape == (self.pT, n)
        assert self.XT.shape == (self.pT, self.pT)
        assert self.rT is None or self.rT.shape == (self.pT,)
        assert self.x0.shape == (n,)


def _c(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------------------
# 2-D constant-velocity vehicle tracking (the paper's Sec. VI-A model).
# ---------------------------------------------------------------------------

def vehicle_model(dt: float = 0.1):
    """F and L of the 2-D constant-velocity model printed in Sec. VI-A:
    state (p_x, p_y, v_x, v_y), control (a_x, a_y)."""
    I2 = np.eye(2)
    Z2 = np.zeros((2, 2))
    F = np.block([[I2, dt * I2], [Z2, I2]])
    L = np.vstack([0.5 * dt * dt * I2, dt * I2])
    return _c(F), _c(L)


def vehicle_reference(T: int, rng: np.random.Generator, noise: float = 0.01) -> np.ndarray:
    """r_k = (sin 0.01k, cos 0.013k) + N(0, noise^2), k = 0..T (row T is r_T)."""
    k = np.arange(T + 1, dtype=np.float64)
    r = np.stack([np.sin(0.01 * k), np.cos(0.013 * k)], axis=1)
    return _c(r + noise * rng.standard_normal(r.shape))


def vehicle(T: int, seed: int = 0, dt: float = 0.1, x_weight: float = 1.0,
            u_weight: float = 0.1, terminal_weight: float = 100.0) -> LQTProblem:
    """Vehicle tracking workload: nx=4, nu=2, p=2.

    F = [[I, dt I], [0, I]], L = [[dt^2/2 I], [dt I]], c = 0, H = [I 0],
    X_k = x_weight I, U_k = u_weight I, terminal H_T = [I 0],
    X_T = terminal_weight I; r_k a sinusoid plus N(0, 0.01^2) noise;
    x_0 ~ N(0, I).  Time-invariant matrices have a leading axis of 1.
    """
    rng = np.random.default_rng(seed)
    F, L = vehicle_model(dt)
    H = np.hstack([np.eye(2), np.zeros((2, 2))])
    r = vehicle_reference(T, rng)
    x0 = rng.standard_normal(4)
    return LQTProblem(
        F=F[None], c=None, L=L[None], U=_c(u_weight * np.eye(2))[None],
        H=_c(H)[None], r=_c(r[:T]), X=_c(x_weight * np.eye(2))[None],
        HT=_c(H), rT=_c(r[T]), XT=_c(terminal_weight * np.eye(2)), x0=_c(x0), T=T)


def paper_tracking(T: int, seed: int = 0, dt: float = 0.1) -> LQTProblem:
    """The cost set-up of Sec. VI-A as printed: reference points every 10th step
    (held in between), X_k = c_k I with c_k = 100 at reference steps and 1e-6
    otherwise, U = 0.1 I, H_T = I_4, X_T = I_4 and a zero terminal velocity.
    The reference points themselves are only shown in a figure, so a seeded
    smooth curve stands in for them."""
    rng = np.random.default_rng(seed)
    F, L = vehicle_model(dt)
    H = np.hstack([np.eye(2), np.zeros((2, 2))])
    n_pts = T // 10 + 1
    s = np.linspace(0.0, 2.0 * math.pi, n_pts)
    pts = np.stack([5.0 * np.cos(s), 5.0 * np.sin(2 * s)], 1) + 0.1 * rng.standard_normal((n_pts, 2))
    k = np.arange(T)
    r = pts[k // 10]
    ck = np.where(k % 10 == 0, 100.0, 1e-6)
    X = ck[:, None, None] * np.eye(2)[None]
    rT = np.concatenate([pts[T // 10], np.zeros(2)])
    x0 = np.array([5.0, 5.0, 0.0, 0.0])
    return LQTProblem(
        F=F[None], c=None, L=L[None], U=_c(0.1 * np.eye(2))[None],
        H=_c(H)[None], r=_c(r), X=_c(X), HT=_c(np.eye(4)), rT=_c(rT),
        XT=_c(np.eye(4)), x0=_c(x0), T=T)


# ---------------------------------------------------------------------------
# Random problems.
# ---------------------------------------------------------------------------

def _stable_dynamics(rng, n, count, radius=1.05, spread=0.05):
    F = np.eye(n)[None] + spread * rng.standard_normal((count, n, n))
    rho = np.abs(np.linalg.eigvals(F)).max(axis=-1)
    scale = np.where(rho > radius, radius / rho, 1.0)
    return F * scale[:, None, None]


def _psd(rng, p, count, rank=None):
    rank = p if rank is None else rank
    B = rng.standard_normal((count, p, rank)) / math.sqrt(max(rank, 1))
    return B @ np.swapaxes(B, 1, 2)


def random_problem(n: int, m: int, p: Optional[int] = None, T: int = 16, seed: int = 0,
                   time_varying: bool = True, with_c: bool = True, pT: Optional[int] = None,
                   x_rank: Optional[int] = None, u_scale: float = 0.1) -> LQTProblem:
    """A random time-varying LQT problem with F_k = I + 0.05 N(0,1) (rescaled to
    spectral radius <= 1.05), L_k ~ N(0, 1/n), X_k = B B^T (PSD, optionally rank
    deficient), U_k = u_scale I + a random SPD part, r_k ~ N(0, 1),
    c_k ~ N(0, 0.1^2)."""
    p = n if p is None else p
    pT = p if pT is None else pT
    rng = np.random.default_rng(seed)
    cnt = T if time_varying else 1
    F = _stable_dynamics(rng, n, cnt)
    L = rng.standard_normal((cnt, n, m)) / math.sqrt(n)
    H = rng.standard_normal((cnt, p, n)) / math.sqrt(n)
    X = _psd(rng, p, cnt, x_rank)
    U = u_scale * np.eye(m)[None] + 0.1 * _psd(rng, m, cnt)
    r = rng.standard_normal((T, p))
    c = 0.1 * rng.standard_normal((cnt, n)) if with_c else None
    HT = rng.standard_normal((pT, n)) / math.sqrt(n)
    XT = _psd(rng, pT, 1)[0]
    rT = rng.standard_normal(pT)
    x0 = rng.standard_normal(n)
    return LQTProblem(F=_c(F), c=None if c is None else _c(c), L=_c(L), U=_c(U), H=_c(H),
                      r=_c(r), X=_c(X), HT=_c(HT), rT=_c(rT), XT=_c(XT), x0=_c(x0), T=T)


def diag_tracking(n: int, T: int, seed: int = 0) -> LQTProblem:
    """Stable random dynamics with m = n/2, H = I, c = 0, X_k = diag(U[0.5, 2]),
    terminal X_T drawn the same way, U = 0.1 I, r_k ~ N(0, 1), x_0 ~ N(0, I)."""
    m = max(n // 2, 1)
    rng = np.random.default_rng(seed)
    F = _stable_dynamics(rng, n, T)
    L = rng.standard_normal((T, n, m)) / math.sqrt(n)
    X = np.zeros((T, n, n))
    idx = np.arange(n)
    X[:, idx, idx] = rng.uniform(0.5, 2.0, (T, n))
    XT = np.diag(rng.uniform(0.5, 2.0, n))
    r = rng.standard_normal((T, n))
    rT = rng.standard_normal(n)
    x0 = rng.standard_normal(n)
    return LQTProblem(F=_c(F), c=None, L=_c(L), U=_c(0.1 * np.eye(m))[None],
                      H=_c(np.eye(n))[None], r=_c(r), X=_c(X), HT=_c(np.eye(n)), rT=_c(rT),
                      XT=_c(XT), x0=_c(x0), T=T)


def scalar_lqr(a: float, b: float, q: float, rho: float, T: int, s_terminal: float,
               x0: float = 1.0) -> LQTProblem:
    """Scalar time-invariant regulator: n = m = p = 1, F = a, L = b, H = 1,
    X = q, U = rho, r = c = 0, terminal weight s_terminal."""
    one = np.ones((1, 1, 1))
    return LQTProblem(F=a * one, c=None, L=b * one, U=rho * one, H=one.copy(), r=None,
                      X=q * one, HT=np.ones((1, 1)), rT=None, XT=np.full((1, 1), s_terminal),
                      x0=np.array([x0], dtype=np.float64), T=T)


def ragged_batch(count: int = 4096, seed: int = 0, sizes=(4, 8, 16), t_min: int = 64,
                 t_max: int = 4096):
    """A ragged batch of `count` diagonal-tracking problems (see diag_tracking):
    n uniform in `sizes`, m = n/2, T uniform in [t_min, t_max], problem i drawn
    with seed (seed, i)."""
    rng = np.random.default_rng(seed)
    ns = rng.choice(np.asarray(sizes), size=count)
    Ts = rng.integers(t_min, t_max + 1, size=count)
    return [diag_tracking(int(n), T=int(T), seed=int(seed) * 1_000_003 + i)
            for i, (n, T) in enumerate(zip(ns, Ts))]


# ---------------------------------------------------------------------------
# Precision study (n = 32, m = 16, ill-conditioned costs).
# ---------------------------------------------------------------------------

def _haar(rng, n, count):
    """Haar-distributed orthogonal matrices: QR of a Gaussian matrix with the
    signs of R's diagonal moved into Q (Mezzadri, Notices AMS 54(5), 2007)."""
    Z = rng.standard_normal((count, n, n))
    Q, R = np.linalg.qr(Z)
    d = np.sign(np.diagonal(R, axis1=1, axis2=2))
    d[d == 0] = 1.0
    return Q * d[:, None, :]


def _cond_spd(rng, n, count, cond):
    """V diag(lam) V^T with V Haar and log10(lam) uniform on [-log10(cond), 0],
    then stretched affinely in log10 so that max/min = cond exactly."""
    V = _haar(rng, n, count)
    e = rng.uniform(-math.log10(cond), 0.0, size=(count, n))
    lo, hi = e.min(axis=1, keepdims=True), e.max(axis=1, keepdims=True)
    e = -math.log10(cond) + math.log10(cond) * (e - lo) / np.maximum(hi - lo, 1e-300)
    lam = 10.0 ** e
    X = (V * lam[:, None, :]) @ np.swapaxes(V, 1, 2)
    return 0.5 * (X + np.swapaxes(X, 1, 2))


def precision_study(T: int = 65536, seed: int = 0, n: int = 32, m: int = 16,
                    cond: float = 1e6, perturb: float = 0.01) -> LQTProblem:
    """F_k = 0.99 Q_k + perturb (u v^T + w z^T) with Q_k Haar orthogonal and
    u, v, w, z ~ N(0, 1/n); X_k = V diag(lam) V^T with cond(X_k) = cond and
    log-uniform eigenvalues; L_k ~ N(0, 1/n), U = 1e-3 I, H = I (p = n),
    c = 0, r_k ~ N(0, 1).  Terminal: H_T = I, X_T drawn like X_k,
    r_T ~ N(0, 1); x_0 ~ N(0, I)."""
    rng = np.random.default_rng(seed)
    Q = _haar(rng, n, T)
    u, v, w, z = (rng.standard_normal((T, n)) / math.sqrt(n) for _ in range(4))
    F = 0.99 * Q + perturb * (u[:, :, None] * v[:, None, :] + w[:, :, None] * z[:, None, :])
    X = _cond_spd(rng, n, T, cond)
    L = rng.standard_normal((T, n, m)) / math.sqrt(n)
    r = rng.standard_normal((T, n))
    XT = _cond_spd(rng, n, 1, cond)[0]
    rT = rng.standard_normal(n)
    x0 = rng.standard_normal(n)
    return LQTProblem(F=_c(F), c=None, L=_c(L), U=_c(1e-3 * np.eye(m))[None],
                      H=_c(np.eye(n))[None], r=_c(r), X=_c(X), HT=_c(np.eye(n)), rT=_c(rT),
                      XT=_c(XT), x0=_c(x0), T=T)


# ---------------------------------------------------------------------------
# Generalised stage cost (Sec. IV-D): cross weights M_k and control offsets s_k.
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class CrossTerms:
    M: Optional[np.ndarray]  # (1|T, p, m) or None (= 0)
    s: Optional[np.ndarray]  # (1|T, m) or None (= 0)

    def astype(self, dtype) -> "CrossTerms":
        def cast(a):
            return None if a is None else np.ascontiguousarray(a, dtype=dtype)

        return CrossTerms(M=cast(self.M), s=cast(self.s))

    def rounded_to(self, dtype) -> "CrossTerms":
        return self.astype(dtype).astype(np.float64)


def _psd_sqrt(A):
    """Symmetric square root of a stack of PSD matrices (eigenvalues clipped at 0)."""
    lam, V = np.linalg.eigh(0.5 * (A + np.swapaxes(A, -1, -2)))
    return (V * np.sqrt(np.maximum(lam, 0.0))[..., None, :]) @ np.swapaxes(V, -1, -2)


def cross_terms(prob: LQTProblem, seed: int = 0, scale: float = 0.5,
                time_varying: bool = True, with_s: bool = True) -> CrossTerms:
    """Cross weights M_k = scale X_k^{1/2} G_k U_k^{1/2} with G_k a Gaussian
    matrix divided by its spectral norm, so that the joint weight
    [[X_k, M_k], [M_k^T, U_k]] >= (1 - scale) blockdiag(X_k, U_k) stays PSD
    (and X_k - M_k U_k^{-1} M_k^T >= (1 - scale^2) X_k); control offsets
    s_k ~ N(0, 1).  With time_varying=False and time-invariant X, U the
    arrays have one row."""
    rng = np.random.default_rng(seed)
    T, m, p = prob.T, prob.m, prob.p
    cnt = T if (time_varying or not prob.time_invariant("X")
                or not prob.time_invariant("U")) else 1
    cnt = max(cnt, 1)
    G = rng.standard_normal((cnt, p, m))
    norms = np.linalg.norm(G, ord=2, axis=(1, 2)) if p > 0 and m > 0 else np.ones(cnt)
    G = G / np.maximum(norms, 1e-300)[:, None, None]
    Xh = _psd_sqrt(np.broadcast_to(prob.X, (cnt, p, p)))
    Uh = _psd_sqrt(np.broadcast_to(prob.U, (cnt, m, m)))
    M = scale * Xh @ G @ Uh
    s = rng.standard_normal((cnt, m)) if with_s else None
    return CrossTerms(M=_c(M), s=None if s is None else _c(s))


# ---------------------------------------------------------------------------
# Unicycle race-track tracking (Sec. VI-E, the nonlinear experiment).
# ---------------------------------------------------------------------------

def stadium_track(sigma, straight: float = 20.0, radius: float = 5.0):
    """Position and unwrapped heading at arc length sigma along a stadium track
    (two straights joined by two half circles, driven counter-clockwise from
    (0, -radius) with heading 0); the heading grows by 2 pi per lap."""
    sigma = np.asarray(sigma, dtype=np.float64)
    per = 2 * straight + 2 * math.pi * radius
    lap = np.floor(sigma / per)
    t = sigma - lap * per
    px = np.empty_like(t)
    py = np.empty_like(t)
    th = np.empty_like(t)
    s1 = t < straight
    s2 = (t >= straight) & (t < straight + math.pi * radius)
    s3 = (t >= straight + math.pi * radius) & (t < 2 * straight + math.pi * radius)
    s4 = t >= 2 * straight + math.pi * radius
    px[s1], py[s1], th[s1] = t[s1], -radius, 0.0
    a2 = (t[s2] - straight) / radius
    px[s2], py[s2], th[s2] = straight + radius * np.sin(a2), -radius * np.cos(a2), a2
    d3 = t[s3] - straight - math.pi * radius
    px[s3], py[s3], th[s3] = straight - d3, radius, math.pi
    a4 = (t[s4] - 2 * straight - math.pi * radius) / radius
    px[s4], py[s4], th[s4] = -radius * np.sin(a4), radius * np.cos(a4), math.pi + a4
    return px, py, th + 2 * math.pi * lap


def unicycle_track(T: int, seed: int = 0, dt: float = 0.1, speed: float = 2.0,
                   ref_every: int = 10, noise: float = 0.01) -> LQTProblem:
    """Cost and initial state of the unicycle experiment (Sec. VI-E): state
    (p_x, p_y, theta, s), control (a, omega); H_k = [I_3 0] (p = 3),
    X_k = diag(100, 100, 1000) at steps with a reference point (every
    `ref_every`-th step) and 1e-6 I otherwise, the same 1e-6 I at k = T;
    U_k = diag(1, 100).  Reference points are positions and headings of a
    stadium track (straights of 20, half circles of radius 5) driven at
    `speed`, plus N(0, noise^2); r_k is held between reference points.
    x_0 = start of the track + N(0, 0.1^2) in position, heading 0, at rest.
    F, L, c are placeholders (identity, zero): the nonlinear solve
    linearises the model itself."""
    rng = np.random.default_rng(seed)
    k = np.arange(T + 1)
    kref = (k // ref_every) * ref_every
    px, py, th = stadium_track(speed * dt * kref)
    r = np.stack([px, py, th], axis=1) + noise * rng.standard_normal((T + 1, 3))
    r = r[(k // ref_every) * ref_every]          # held between reference points
    is_ref = (k % ref_every) == 0
    X = np.zeros((T + 1, 3, 3))
    X[:, 0, 0] = np.where(is_ref, 100.0, 1e-6)
    X[:, 1, 1] = X[:, 0, 0]
    X[:, 2, 2] = np.where(is_ref, 1000.0, 1e-6)
    X[T] = 1e-6 * np.eye(3)
    H = np.hstack([np.eye(3), np.zeros((3, 1))])
    x0 = np.array([0.0, -5.0, 0.0, 0.0])
    x0[:2] += 0.1 * rng.standard_normal(2)
    return LQTProblem(F=_c(np.eye(4))[None], c=None, L=_c(np.zeros((4, 2)))[None],
                      U=_c(np.diag([1.0, 100.0]))[None], H=_c(H)[None], r=_c(r[:T]),
                      X=_c(X[:T]), HT=_c(H), rT=_c(r[T]), XT=_c(X[T]), x0=_c(x0), T=T)
