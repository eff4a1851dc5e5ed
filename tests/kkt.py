"""Dense KKT brute force for the LQT quadratic program of eq. LQT_problem.

Independent of the oracle: the whole problem is written as one equality-
constrained quadratic program and solved by a single dense LAPACK solve.

Variables z = (u_k, ..., u_{T-1}, x_{k+1}, ..., x_T) with x_k fixed;
cost  sum_{t=k}^{T-1} 1/2 (H_t x_t - r_t)^T X_t (H_t x_t - r_t) + 1/2 u_t^T U_t u_t
      + 1/2 (H_T x_T - r_T)^T X_T (H_T x_T - r_T);
constraints x_{t+1} = F_t x_t + c_t + L_t u_t.

With a cross weight M_t (p x m) and a control offset s_t (m) the stage cost is
that of eq. generalised_cost (Sec. IV-D):
1/2 e^T X e + e^T M (u - s) + 1/2 (u - s)^T U (u - s), e = H_t x_t - r_t,
expanded term by term into the same quadratic program.
"""
import numpy as np


def _step(a, t):
    if a is None:
        return None
    return a[0] if a.shape[0] == 1 else a[t]


def solve_from(prob, k, xk, M=None, s=None):
    """Optimal (u_k..u_{T-1}, x_k..x_T, cost) of the tail problem started at x_k
    (with the generalised stage cost when M or s is given)."""
    n, m, T = prob.n, prob.m, prob.T
    N = T - k
    nu, nx = N * m, N * n
    nz = nu + nx
    P = np.zeros((nz, nz))
    q = np.zeros(nz)
    const = 0.0

    def uidx(t):
        return slice((t - k) * m, (t - k + 1) * m)

    def xidx(t):  # t in k+1..T
        o = nu + (t - k - 1) * n
        return slice(o, o + n)

    # stage costs
    for t in range(k, T):
        H, X, U = _step(prob.H, t), _step(prob.X, t), _step(prob.U, t)
        r = _step(prob.r, t)
        r = np.zeros(H.shape[0]) if r is None else r
        P[uidx(t), uidx(t)] += U
        if t == k:
            e = H @ xk - r
            const += 0.5 * e @ X @ e
        else:
            P[xidx(t), xidx(t)] += H.T @ X @ H
            q[xidx(t)] -= H.T @ X @ r
            const += 0.5 * r @ X @ r
        Mt = _step(M, t)
        st = _step(s, t)
        st = np.zeros(m) if st is None else st
        # 1/2 (u - s)^T U (u - s) beyond 1/2 u^T U u: -s^T U u + 1/2 s^T U s
        q[uidx(t)] -= U @ st
        const += 0.5 * st @ U @ st
        if Mt is not None:
            # (H x - r)^T M (u - s) = x^T H^T M u - x^T H^T M s - r^T M u + r^T M s
            if t == k:
                e = H @ xk - r
                q[uidx(t)] += Mt.T @ e
                const -= e @ Mt @ st
            else:
                P[xidx(t), uidx(t)] += H.T @ Mt
                P[uidx(t), xidx(t)] += Mt.T @ H
                q[xidx(t)] -= H.T @ Mt @ st
                q[uidx(t)] -= Mt.T @ r
                const += r @ Mt @ st
    rT = np.zeros(prob.pT) if prob.rT is None else prob.rT
    if N == 0:
        e = prob.HT @ xk - rT
        return np.zeros((0, m)), xk[None].copy(), 0.5 * e @ prob.XT @ e
    P[xidx(T), xidx(T)] += prob.HT.T @ prob.XT @ prob.HT
    q[xidx(T)] -= prob.HT.T @ prob.XT @ rT
    const += 0.5 * rT @ prob.XT @ rT

    # dynamics: x_{t+1} - F x_t - L u_t = c_t
    E = np.zeros((nx, nz))
    e = np.zeros(nx)
    for t in range(k, T):
        F, L = _step(prob.F, t), _step(prob.L, t)
        c = _step(prob.c, t)
        c = np.zeros(n) if c is None else c
        row = slice((t - k) * n, (t - k + 1) * n)
        E[row, xidx(t + 1)] = np.eye(n)
        E[row, uidx(t)] = -L
        if t == k:
            e[row] = F @ xk + c
        else:
            E[row, xidx(t)] = -F
            e[row] = c

    KKT = np.block([[P, E.T], [E, np.zeros((nx, nx))]])
    rhs = np.concatenate([-q, e])
    sol = np.linalg.solve(KKT, rhs)
    z = sol[:nz]
    u = z[:nu].reshape(N, m)
    x = np.vstack([xk[None], z[nu:].reshape(N, n)])
    cost = 0.5 * z @ P @ z + q @ z + const
    return u, x, cost


def value_function(prob, k, M=None, s=None):
    """(S_k, v_k, K_k, ff_k) of the tail problem at k, read off the brute-force
    solutions: V_k(x) = z + 1/2 x^T S_k x - v_k^T x is quadratic, so its Hessian
    and gradient come exactly from costs at 0, +-e_i and e_i + e_j; the first
    control u_k(x) = -K_k x + ff_k is affine in x."""
    n = prob.n
    I = np.eye(n)
    V0 = solve_from(prob, k, np.zeros(n), M, s)
    Vp = [solve_from(prob, k, I[i], M, s) for i in range(n)]
    Vm = [solve_from(prob, k, -I[i], M, s) for i in range(n)]
    S = np.zeros((n, n))
    v = np.zeros(n)
    for i in range(n):
        S[i, i] = Vp[i][2] + Vm[i][2] - 2 * V0[2]
        v[i] = -(Vp[i][2] - Vm[i][2]) / 2
        for j in range(i + 1, n):
            Vij = solve_from(prob, k, I[i] + I[j], M, s)[2]
            S[i, j] = S[j, i] = Vij - Vp[i][2] - Vp[j][2] + V0[2]
    if k < prob.T:
        ff = V0[0][0]
        K = np.stack([-(Vp[i][0][0] - ff) for i in range(n)], axis=1)
    else:
        ff = K = None
    return S, v, K, ff


def total_cost(prob, u, M=None, s=None):
    """Cost of eq. LQT_problem (eq. generalised_cost stages when M or s is
    given) for a control sequence u (T, m) from x_0."""
    n, T = prob.n, prob.T
    x = prob.x0.copy()
    J = 0.0
    for t in range(T):
        H, X, U = _step(prob.H, t), _step(prob.X, t), _step(prob.U, t)
        r = _step(prob.r, t)
        r = np.zeros(H.shape[0]) if r is None else r
        e = H @ x - r
        st = _step(s, t)
        du = u[t] - (0 if st is None else st)
        J += 0.5 * e @ X @ e + 0.5 * du @ U @ du
        Mt = _step(M, t)
        if Mt is not None:
            J += e @ Mt @ du
        c = _step(prob.c, t)
        x = _step(prob.F, t) @ x + (0 if c is None else c) + _step(prob.L, t) @ u[t]
    rT = np.zeros(prob.pT) if prob.rT is None else prob.rT
    e = prob.HT @ x - rT
    return J + 0.5 * e @ prob.XT @ e
