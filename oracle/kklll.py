"""ORACLE -- test infrastructure only.  Algorithm KKLLL (Section 2.3) in fp64.

For a 0/1 pattern B (the pattern matrix of Section 3: b_ij = 1 where
a_ij != 0), every nonzero entry is replaced by a cube root of unity drawn
uniformly and independently, and X = det(W) * conj(det(W)) = |det W|^2 is an
unbiased estimate of per(B) (the paper's Theorem).  The approximate
permanent of a job is the mean of X over T trials; the paper uses T of about
n^2 (Table T5 and T8 footnotes).

The draws come from a counter-based generator so that any implementation can
reproduce them: SplitMix64's output function (Steele, Lea and Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014) applied to

    x = seed ^ (job * 0xD1B54A32D192ED03) ^ (trial * 0xABC98388FB8FAC03)
             ^ (e * 0x8CB92BA72F3D8DD7)        (mod 2^64)

with e = i*m + j the entry's row-major index in the m x m job; the cube
root index is floor(3 * (h >> 32) / 2^32).
"""
from __future__ import annotations

import itertools
import math

import numpy as np

M64 = (1 << 64) - 1
K_JOB = 0xD1B54A32D192ED03
K_TRIAL = 0xABC98388FB8FAC03
K_ENTRY = 0x8CB92BA72F3D8DD7
OMEGA = (complex(1.0, 0.0), complex(-0.5, math.sqrt(3.0) / 2.0),
         complex(-0.5, -math.sqrt(3.0) / 2.0))


def splitmix64_mix(z: int) -> int:
    """SplitMix64: add the golden gamma, then the two xor-shift-multiply
    rounds and a final xor-shift of the published generator."""
    z = (z + 0x9E3779B97F4A7C15) & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def kklll_choice(seed: int, job: int, trial: int, e: int) -> int:
    """Index in {0, 1, 2} of the cube root drawn for entry e of trial t."""
    x = (seed ^ ((job * K_JOB) & M64) ^ ((trial * K_TRIAL) & M64) ^ ((e * K_ENTRY) & M64)) & M64
    h = splitmix64_mix(x)
    return ((h >> 32) * 3) >> 32


def det_partial_pivot(w: np.ndarray):
    """Gaussian elimination with partial pivoting on |z| (the first row of
    largest modulus wins a tie).  Returns (log |det|^2, zero_flag)."""
    a = np.array(w, dtype=np.complex128, copy=True)
    m = a.shape[0]
    logabs2 = 0.0
    for k in range(m):
        mags = np.abs(a[k:, k])
        p = k + int(np.argmax(mags))
        if mags[p - k] == 0.0:
            return -math.inf, True
        if p != k:
            a[[k, p]] = a[[p, k]]
        piv = a[k, k]
        logabs2 += math.log(piv.real * piv.real + piv.imag * piv.imag)
        if k + 1 < m:
            f = a[k + 1:, k] / piv
            a[k + 1:, k + 1:] -= np.outer(f, a[k, k + 1:])
    return logabs2, False


def _trial_matrix(pattern: np.ndarray, seed: int, job: int, trial: int) -> np.ndarray:
    m = pattern.shape[0]
    w = np.zeros((m, m), dtype=np.complex128)
    for i in range(m):
        for j in range(m):
            if pattern[i, j]:
                w[i, j] = OMEGA[kklll_choice(seed, job, trial, i * m + j)]
    return w


def kklll_trial_log_abs2(a, seed: int, job: int, trial: int) -> float:
    """log |det W|^2 for one trial on the pattern of ``a``."""
    pattern = np.asarray(a) != 0
    return det_partial_pivot(_trial_matrix(pattern, seed, job, trial))[0]


def kklll_log_ap(a, seed: int, job: int, trials: int | None = None) -> float:
    """log of the KKLLL approximate permanent: log mean_t |det W_t|^2 over
    ``trials`` trials (default m^2).  -inf when every trial is singular."""
    pattern = np.asarray(a) != 0
    m = pattern.shape[0]
    if m == 0:
        return 0.0
    t_count = m * m if not trials else int(trials)
    logs = [det_partial_pivot(_trial_matrix(pattern, seed, job, t))[0] for t in range(t_count)]
    top = max(logs)
    if top == -math.inf:
        return -math.inf
    s = sum(math.exp(v - top) for v in logs if v != -math.inf)
    return top + math.log(s / t_count)


def kklll_exact_mean(a) -> float:
    """E[|det W|^2] by enumerating all 3^nnz choices (tiny patterns only).

    The paper's Theorem states this equals per(B)."""
    pattern = np.asarray(a) != 0
    m = pattern.shape[0]
    pos = [(i, j) for i in range(m) for j in range(m) if pattern[i, j]]
    if len(pos) > 12:
        raise ValueError("exact enumeration is for nnz <= 12")
    total = 0.0
    for choice in itertools.product(range(3), repeat=len(pos)):
        w = np.zeros((m, m), dtype=np.complex128)
        for (i, j), c in zip(pos, choice):
            w[i, j] = OMEGA[c]
        d = np.linalg.det(w)
        total += (d * d.conjugate()).real
    return total / 3 ** len(pos)
