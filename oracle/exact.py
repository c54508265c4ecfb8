"""Exact master-equation evaluators for tiny lattices (L <= 10): the expected density of
one sample, computed by evolving the full probability vector over all 2^L configurations.

TEST INFRASTRUCTURE ONLY (used by tests/ to pin the Monte Carlo oracle).

Two discrete-time chains, both written from the paper (Schram, arXiv 1301.6082):

* ``rs_*`` -- Alg. 1 (Sec. 2): one attempt picks a bond (i, i+1) with
  probability w_i, diffuses with probability P_D, else on an occupied pair annihilates with
  probability P_P or creates a particle at i-1 / i+2 with probability 1/2 each.  One attempt
  is 1/L MCS; t MCS are t*L attempts.  This is the discrete operator A = sum_i w_i K_i, not
  exp(Q t): the two differ by O(1/L).

* ``sched_*`` -- the random-phase 3-site window schedule (R2 of the design): sub-step =
  sum over phases phi (weight w_phi) of the product of independent 3-site kernels on the
  windows (phi+3k, phi+3k+1, phi+3k+2), k < K = floor(L/3); leftover sites idle.  MCS time t
  is sub-step ceil(t*L/K).  The same with windows of n+1 sites for the n-tuple processes
  (TCPD n = 3, QCPD n = 4; R14).

Probabilities come from the integer thresholds exactly: P_D = T_D/2^32,
P_A = (T_DA - T_D)/2^32, P_F = 1 - T_DA/2^32 (window form); P_P = T_P/2^32 (Alg. 1 form).
Site / phase weights w_j = (ceil((j+1) 2^32/L) - ceil(j 2^32/L)) / 2^32 -- the exact law of
floor(x*L/2^32) for a uniform 32-bit x.
"""
from __future__ import annotations

import numpy as np

TWO32 = 1 << 32


def index_weights(L: int) -> np.ndarray:
    """Exact law of floor(x*L/2^32), x uniform on [0, 2^32)."""
    def ceil_div(a, b):
        return -((-a) // b)
    cnt = [ceil_div((j + 1) * TWO32, L) - ceil_div(j * TWO32, L) for j in range(L)]
    assert sum(cnt) == TWO32
    return np.array(cnt, dtype=np.float64) / TWO32


def _apply_local(v: np.ndarray, L: int, sites, K: np.ndarray) -> np.ndarray:
    """Apply a kernel K[new, old] on the given sites (bit order: sites[0] is the most
    significant local bit) to a probability vector indexed by configurations x (bit i of x =
    occupation of site i)."""
    m = len(sites)
    t = v.reshape((2,) * L)
    axes = [L - 1 - s for s in sites]  # C-order axis of bit s
    t = np.moveaxis(t, axes, list(range(m)))
    sh = t.shape
    t = K @ t.reshape(1 << m, -1)
    t = t.reshape(sh)
    t = np.moveaxis(t, list(range(m)), axes)
    return np.ascontiguousarray(t).reshape(-1)


def window_kernel(pD: float, pA: float) -> np.ndarray:
    """8x8 kernel of one window (a, b, c); local index a*4 + b*2 + c.
    Orientation o (1/2 each) picks bond (a,b)->target c or bond (b,c)->target a; then
    diffusion (pD) swaps the bond, annihilation (pA) clears an occupied bond, fission
    (1-pD-pA) fills the target next to an occupied bond."""
    pF = 1.0 - pD - pA
    K = np.zeros((8, 8))
    for old in range(8):
        for o in (0, 1):
            for cls, pr in (("D", pD), ("A", pA), ("F", pF)):
                s = [(old >> 2) & 1, (old >> 1) & 1, old & 1]
                qi, ti = (2, 0) if o else (0, 2)
                if cls == "D":
                    s[1], s[qi] = s[qi], s[1]
                elif s[1] == 1 and s[qi] == 1:
                    if cls == "A":
                        s[1] = s[qi] = 0
                    else:
                        s[ti] = 1
                new = s[0] * 4 + s[1] * 2 + s[2]
                K[new, old] += 0.5 * pr
    return K


def tuple_window_kernel(pD: float, pA: float, n: int) -> np.ndarray:
    """Kernel of one window of W = n+1 sites for the n-tuple process (R14): local index bit
    W-1-j is site w_j.  Orientation o (1/2 each): o = 0 takes the tuple w_0..w_{n-1}, the
    bond (w_0, w_1) and the target w_n; o = 1 the tuple w_1..w_n, the bond (w_1, w_2) and the
    target w_0.  Diffusion (pD) swaps the bond; otherwise, on a fully occupied tuple,
    annihilation (pA) empties it and fission (1-pD-pA) fills the target."""
    W = n + 1
    pF = 1.0 - pD - pA
    K = np.zeros((1 << W, 1 << W))
    for old in range(1 << W):
        s0 = [(old >> (W - 1 - j)) & 1 for j in range(W)]
        for o in (0, 1):
            tup = list(range(1, W)) if o else list(range(0, n))
            b0 = tup[0]
            tgt = 0 if o else n
            for cls, pr in (("D", pD), ("A", pA), ("F", pF)):
                s = list(s0)
                if cls == "D":
                    s[b0], s[b0 + 1] = s[b0 + 1], s[b0]
                elif all(s[j] == 1 for j in tup):
                    if cls == "A":
                        for j in tup:
                            s[j] = 0
                    else:
                        s[tgt] = 1
                new = sum(b << (W - 1 - j) for j, b in enumerate(s))
                K[new, old] += 0.5 * pr
    return K


def sched_substep(v: np.ndarray, L: int, t_d: int, t_da: int, phase_w=None, n: int = 2) -> np.ndarray:
    """One sub-step of the window schedule: windows of W = n+1 sites (n = 2: the PCPD's
    3-site windows with the kernel above), K = floor(L/W) of them at each phase."""
    pD = t_d / TWO32
    pA = (t_da - t_d) / TWO32
    W = n + 1
    Kw = window_kernel(pD, pA) if n == 2 else tuple_window_kernel(pD, pA, n)
    nwin = L // W
    w = index_weights(L) if phase_w is None else phase_w
    out = np.zeros_like(v)
    for phi in range(L):
        u = v
        for k in range(nwin):
            sites = [(phi + W * k + r) % L for r in range(W)]
            u = _apply_local(u, L, sites, Kw)
        out += w[phi] * u
    return out


def bond_kernel_alg1(pD: float, pP: float) -> np.ndarray:
    """16x16 kernel of Alg. 1 on sites (i-1, i, i+1, i+2) given that bond (i, i+1) is picked
    (local index bit 3 = i-1 ... bit 0 = i+2)."""
    K = np.zeros((16, 16))
    for old in range(16):
        lo, qi, qi1, hi = (old >> 3) & 1, (old >> 2) & 1, (old >> 1) & 1, old & 1
        outs = []
        # r1 < d: swap q_i, q_{i+1}
        outs.append((pD, (lo, qi1, qi, hi)))
        if qi == 1 and qi1 == 1:
            outs.append(((1 - pD) * pP, (lo, 0, 0, hi)))                 # annihilation
            outs.append(((1 - pD) * (1 - pP) * 0.5, (1, qi, qi1, hi)))   # fission low
            outs.append(((1 - pD) * (1 - pP) * 0.5, (lo, qi, qi1, 1)))   # fission high
        else:
            outs.append((1 - pD, (lo, qi, qi1, hi)))
        for pr, (a, b, c, d) in outs:
            K[a * 8 + b * 4 + c * 2 + d, old] += pr
    return K


def rs_attempt(v: np.ndarray, L: int, t_d: int, t_p: int, site_w=None) -> np.ndarray:
    """One Alg. 1 attempt; needs L >= 4 so that i-1, i, i+1, i+2 are distinct (L = 3 is
    handled by rs_attempt_small)."""
    if L < 4:
        return rs_attempt_small(v, L, t_d, t_p, site_w)
    K = bond_kernel_alg1(t_d / TWO32, t_p / TWO32)
    w = index_weights(L) if site_w is None else site_w
    out = np.zeros_like(v)
    for i in range(L):
        sites = [(i - 1) % L, i, (i + 1) % L, (i + 2) % L]
        out += w[i] * _apply_local(v, L, sites, K)
    return out


def rs_attempt_small(v, L, t_d, t_p, site_w=None):
    """Alg. 1 on rings where i-1 and i+2 coincide (L = 3): apply the rule literally on the
    configuration."""
    pD, pP = t_d / TWO32, t_p / TWO32
    w = index_weights(L) if site_w is None else site_w
    n = 1 << L
    out = np.zeros_like(v)
    for x in range(n):
        if v[x] == 0.0:
            continue
        for i in range(L):
            q = [(x >> s) & 1 for s in range(L)]
            i1, im, i2 = (i + 1) % L, (i - 1) % L, (i + 2) % L
            res = []
            qs = q.copy(); qs[i], qs[i1] = qs[i1], qs[i]
            res.append((pD, qs))
            if q[i] == 1 and q[i1] == 1:
                qa = q.copy(); qa[i] = qa[i1] = 0
                ql = q.copy(); ql[im] = 1
                qh = q.copy(); qh[i2] = 1
                res += [((1 - pD) * pP, qa), ((1 - pD) * (1 - pP) * 0.5, ql),
                        ((1 - pD) * (1 - pP) * 0.5, qh)]
            else:
                res.append((1 - pD, q))
            for pr, qq in res:
                y = sum(b << s for s, b in enumerate(qq))
                out[y] += v[x] * w[i] * pr
    return out


def pair_occupation(L: int) -> np.ndarray:
    """Occupied nearest-neighbour pairs (i, i+1 mod L) of every configuration."""
    x = np.arange(1 << L)
    rot = ((x >> 1) | ((x & 1) << (L - 1)))
    both = x & rot
    return np.array([bin(int(i)).count("1") for i in both], dtype=np.float64)


def sched_observable(L: int, t_d: int, t_da: int, rec_sub, obs: np.ndarray, mode: str = "full"):
    """Exact mean and variance of a per-configuration observable (divided by L) after each
    sub-step count in rec_sub."""
    v = start_vector(L, mode)
    w = index_weights(L)
    mean, var, n = [], [], 0
    for r in rec_sub:
        while n < r:
            v = sched_substep(v, L, t_d, t_da, w)
            n += 1
        m1 = float(v @ obs) / L
        m2 = float(v @ (obs * obs)) / (L * L)
        mean.append(m1)
        var.append(max(0.0, m2 - m1 * m1))
    return np.array(mean), np.array(var)


def occupation(L: int) -> np.ndarray:
    x = np.arange(1 << L)
    return np.array([bin(int(i)).count("1") for i in x], dtype=np.float64)


def start_vector(L: int, mode: str = "full") -> np.ndarray:
    v = np.zeros(1 << L)
    if mode == "full":
        v[(1 << L) - 1] = 1.0
    elif mode == "half":
        v[:] = 1.0 / (1 << L)
    else:
        raise ValueError(mode)
    return v


def sched_moments(L: int, t_d: int, t_da: int, rec_sub, mode: str = "full", tuple_n: int = 2):
    """Exact E[rho] and Var[rho] of one sample after each sub-step count in rec_sub
    (tuple_n: 2 PCPD, 3 TCPD, 4 QCPD)."""
    occ = occupation(L)
    v = start_vector(L, mode)
    w = index_weights(L)
    mean, var, n = [], [], 0
    for r in rec_sub:
        while n < r:
            v = sched_substep(v, L, t_d, t_da, w, tuple_n)
            n += 1
        m1 = float(v @ occ) / L
        m2 = float(v @ (occ * occ)) / (L * L)
        mean.append(m1)
        var.append(max(0.0, m2 - m1 * m1))
    return np.array(mean), np.array(var)


def sched_density(L: int, t_d: int, t_da: int, rec_sub, mode: str = "full") -> np.ndarray:
    """Exact E[rho] after each sub-step count in rec_sub (sorted)."""
    return sched_moments(L, t_d, t_da, rec_sub, mode)[0]


def rs_moments(L: int, t_d: int, t_p: int, rec_att, mode: str = "full"):
    """Exact E[rho] and Var[rho] of one sample after each attempt count in rec_att."""
    occ = occupation(L)
    v = start_vector(L, mode)
    w = index_weights(L)
    mean, var, m = [], [], 0
    for r in rec_att:
        while m < r:
            v = rs_attempt(v, L, t_d, t_p, w)
            m += 1
        m1 = float(v @ occ) / L
        m2 = float(v @ (occ * occ)) / (L * L)
        mean.append(m1)
        var.append(max(0.0, m2 - m1 * m1))
    return np.array(mean), np.array(var)


def rs_density(L: int, t_d: int, t_p: int, rec_att, mode: str = "full") -> np.ndarray:
    """Exact E[rho] after each attempt count in rec_att (sorted)."""
    return rs_moments(L, t_d, t_p, rec_att, mode)[0]
