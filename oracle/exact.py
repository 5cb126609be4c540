"""Exact master-equation enumeration for tiny lattices (test infrastructure).

States are the 2^n bit patterns of n lattice bits with a fixed particle count
(n = L for one ring, n = 2L for the two-lane model, where bit i is lane A's
site i and bit L + i lane B's site i).  Every update step of the method is a
row-stochastic matrix on that space, built from its definition:

* one attempt on bond b: the bond kernel K_b (paper sec. 2.1: a particle
  hops right with p_i into an empty right neighbour, left with q_{i+1});
* serial RSU sweep: (1/B sum_b K_b)^B for B bonds (L or 2L attempts);
* continuous-time generator: Q = sum_b (K_b - I);
* a domain with m bonds running a Poisson(m) number of uniform attempts:
  sum_k e^{-m} m^k / k! (M_dom)^k = exp(sum_{b in dom} (K_b - I));
* the two-phase domain sweep: the average over the 2D offsets o of
  exp(Q_even(o)) exp(Q_odd(o)), the domains of one phase being disjoint;
* the two-sub-lattice SCA sweep (paper sec. 2.1): the product of the even
  bonds' kernels, then of the odd bonds' kernels; two lanes (sec. 3): with
  the one-directional lane changes after each phase;
* the lane-change pass of the two-lane model: a product of independent
  per-site swaps with probability omega where exactly one lane is occupied.

Row-vector convention: a distribution pi evolves as pi @ A.
"""
from __future__ import annotations

from fractions import Fraction
from itertools import combinations

import numpy as np
from scipy.linalg import expm


class Space:
    """Bit patterns of ``nbits`` bits with ``N`` ones (ring: nbits = L)."""

    def __init__(self, L: int, N: int, lanes: int = 1):
        self.L, self.N, self.lanes = L, N, lanes
        nbits = L * lanes
        self.states = [sum(1 << b for b in c) for c in combinations(range(nbits), N)]
        self.index = {x: k for k, x in enumerate(self.states)}
        self.n = len(self.states)

    def bit(self, x: int, lane: int, i: int) -> int:
        return (x >> (lane * self.L + i % self.L)) & 1

    def flip(self, x: int, lane: int, i: int) -> int:
        return x ^ (1 << (lane * self.L + i % self.L))

    # -- one-attempt kernels ------------------------------------------------
    def bond_kernel(self, lane: int, b: int, p_right: float, q_left: float) -> np.ndarray:
        """One attempt on bond (b, b+1) of ``lane``: 10 -> 01 with p_right,
        01 -> 10 with q_left."""
        K = np.zeros((self.n, self.n))
        for k, x in enumerate(self.states):
            a, c = self.bit(x, lane, b), self.bit(x, lane, b + 1)
            y = self.flip(self.flip(x, lane, b), lane, b + 1)
            if a == 1 and c == 0:
                K[k, self.index[y]] += p_right
                K[k, k] += 1 - p_right
            elif a == 0 and c == 1:
                K[k, self.index[y]] += q_left
                K[k, k] += 1 - q_left
            else:
                K[k, k] += 1
        return K

    def turning_kernel(self, turning_sites, omega, omega_ba=None) -> np.ndarray:
        """Two lanes: at each turning site with exactly one lane occupied, the
        particle moves to the other lane with probability omega (a number or a
        per-site dict; with ``omega_ba`` the moves from lane B use that one)."""
        T = np.eye(self.n)
        for i in turning_sites:
            Ti = np.zeros((self.n, self.n))
            for k, x in enumerate(self.states):
                if self.bit(x, 0, i) != self.bit(x, 1, i):
                    y = self.flip(self.flip(x, 0, i), 1, i)
                    w = omega if self.bit(x, 0, i) or omega_ba is None else omega_ba
                    w = w[i] if isinstance(w, dict) else w
                    Ti[k, self.index[y]] += w
                    Ti[k, k] += 1 - w
                else:
                    Ti[k, k] += 1
            T = T @ Ti
        return T

    def lane_change_kernel(self, turning_sites, omega, src: int) -> np.ndarray:
        """Two lanes, one direction: at each turning site whose lane `src` is
        occupied and other lane empty, the particle moves across with
        probability omega (a number or a per-site dict)."""
        T = np.eye(self.n)
        for i in turning_sites:
            w = omega[i] if isinstance(omega, dict) else omega
            Ti = np.zeros((self.n, self.n))
            for k, x in enumerate(self.states):
                if self.bit(x, src, i) == 1 and self.bit(x, 1 - src, i) == 0:
                    y = self.flip(self.flip(x, 0, i), 1, i)
                    Ti[k, self.index[y]] += w
                    Ti[k, k] += 1 - w
                else:
                    Ti[k, k] += 1
            T = T @ Ti
        return T

    # -- observables ---------------------------------------------------------
    def w2(self, lane: int = 0) -> np.ndarray:
        """W^2 of Eq. (W) per state, heights h_i = sum_{j<=i} (2 n_j - 1)."""
        out = np.zeros(self.n)
        L = self.L
        for k, x in enumerate(self.states):
            h, s1, s2 = 0, 0, 0
            for i in range(L):
                h += 2 * self.bit(x, lane, i) - 1
                s1 += h
                s2 += h * h
            out[k] = float(Fraction(L * s2 - s1 * s1, L * L))
        return out

    def flat_alt(self) -> np.ndarray:
        """Delta distribution on the alternating 1010... start (site 0 occupied)
        in every lane."""
        x = 0
        for lane in range(self.lanes):
            for i in range(0, self.L, 2):
                x |= 1 << (lane * self.L + i)
        v = np.zeros(self.n)
        v[self.index[x]] = 1.0
        return v


class RingModel:
    """One ASEP ring: per-site right rates p[i] and left rates q[i]; bond b
    uses p[b] for the right hop and q[b+1] for the left hop."""

    def __init__(self, L: int, N: int, p, q):
        self.sp = Space(L, N, 1)
        self.L = L
        p = [p] * L if np.isscalar(p) else list(p)
        q = [q] * L if np.isscalar(q) else list(q)
        self.K = [self.sp.bond_kernel(0, b, p[b], q[(b + 1) % L]) for b in range(L)]
        self.I = np.eye(self.sp.n)

    def rsu_sweep(self) -> np.ndarray:
        M = sum(self.K) / self.L
        return np.linalg.matrix_power(M, self.L)

    def generator(self) -> np.ndarray:
        return sum(K - self.I for K in self.K)

    def sca_sweep(self) -> np.ndarray:
        """The paper's two-sub-lattice SCA sweep: one attempt on every even
        bond, then one on every odd bond (disjoint bonds, so each phase is a
        product of commuting kernels); even first."""
        E, O = self.I, self.I
        for b in range(0, self.L, 2):
            E = E @ self.K[b]
        for b in range(1, self.L, 2):
            O = O @ self.K[b]
        return E @ O

    def domain_sweep(self, D: int) -> np.ndarray:
        L = self.L
        assert L % (2 * D) == 0
        total = np.zeros_like(self.I)
        for o in range(2 * D):
            A = self.I
            for phase in (0, 1):
                Q = np.zeros_like(self.I)
                for g in range(L // (2 * D)):
                    base = o + 2 * D * g + phase * D
                    for j in range(D):
                        Q += self.K[(base + j) % L] - self.I
                A = A @ expm(Q)
            total += A
        return total / (2 * D)

    def current_per_attempt_vector(self, p, q) -> np.ndarray:
        """Expected net right hops summed over bonds for one attempt on each
        bond, per state (homogeneous rates)."""
        sp = self.sp
        out = np.zeros(sp.n)
        for k, x in enumerate(sp.states):
            for b in range(self.L):
                a, c = sp.bit(x, 0, b), sp.bit(x, 0, b + 1)
                if a == 1 and c == 0:
                    out[k] += p
                elif a == 0 and c == 1:
                    out[k] -= q
        return out


class TwoLaneModel:
    """Two rings: lane A hops right with pA, lane B hops left with pB; lane
    changes at ``turning_sites`` with probability omega once per sweep (A -> B
    with ``omega``, B -> A with ``omega_ba`` when given; either may be a
    per-site dict, the paper's crossing probabilities u_i and v_i)."""

    def __init__(self, L: int, N: int, pA: float, pB: float, turning_sites, omega, omega_ba=None):
        self.sp = Space(L, N, 2)
        self.L = L
        self.KA = [self.sp.bond_kernel(0, b, pA, 0.0) for b in range(L)]
        self.KB = [self.sp.bond_kernel(1, b, 0.0, pB) for b in range(L)]
        ba = omega if omega_ba is None else omega_ba
        self.T = self.sp.turning_kernel(list(turning_sites), omega, ba)
        self.TAB = self.sp.lane_change_kernel(list(turning_sites), omega, 0)
        self.TBA = self.sp.lane_change_kernel(list(turning_sites), ba, 1)
        self.I = np.eye(self.sp.n)

    def rsu_sweep(self) -> np.ndarray:
        M = (sum(self.KA) + sum(self.KB)) / (2 * self.L)
        return np.linalg.matrix_power(M, 2 * self.L) @ self.T

    def domain_sweep(self, D: int) -> np.ndarray:
        L = self.L
        total = np.zeros_like(self.I)
        for o in range(2 * D):
            A = self.I
            for phase in (0, 1):
                Q = np.zeros_like(self.I)
                for g in range(L // (2 * D)):
                    base = o + 2 * D * g + phase * D
                    for j in range(D):
                        b = (base + j) % L
                        Q += (self.KA[b] - self.I) + (self.KB[b] - self.I)
                A = A @ expm(Q)
            total += A
        return (total / (2 * D)) @ self.T

    def sca_sweep(self) -> np.ndarray:
        """The two-lane SCA sweep (paper sec. 3, five steps): even bonds of
        both lanes, A -> B lane changes, odd bonds of both lanes (the closing
        bonds with them), B -> A lane changes."""
        E, O = self.I, self.I
        for b in range(0, self.L, 2):
            E = E @ self.KA[b] @ self.KB[b]
        for b in range(1, self.L, 2):
            O = O @ self.KA[b] @ self.KB[b]
        return E @ self.TAB @ O @ self.TBA


def stationary(A: np.ndarray) -> np.ndarray:
    """Left Perron vector of a stochastic matrix (pi A = pi, sum pi = 1)."""
    w, v = np.linalg.eig(A.T)
    k = int(np.argmin(np.abs(w - 1.0)))
    pi = np.real(v[:, k])
    return pi / pi.sum()
