"""Seeded synthetic inputs shared by the CUDA library's callers and the CPU oracle.

This module holds random draws only -- none of the performance-modeling
method's arithmetic -- so that both sides can be fed identical inputs without
sharing any code that computes a result.  Every generator is a NumPy PCG64
stream keyed by an integer seed; the workload recipes (shapes, sizes, value
distributions) follow the paper's workloads:

  * matmul: A, B ~ U[-1, 1] fp32 (Section "Matrix Multiplication");
  * DG differentiation: D, u ~ N(0, 1) fp32 (Section "DG");
  * five-point stencil: u ~ U[-1, 1] fp32 (Section "Finite Differences");
  * calibration suite: values ~ U[-1, 1] (Section "Measurement Kernel Design");
  * fits: design matrices of positive integer feature counts, positive
    parameters drawn log-uniformly, relative noise eps ~ N(0, 1).
"""
import numpy as np


def rng(seed):
    return np.random.Generator(np.random.PCG64(int(seed)))


def uniform(shape, seed, lo=-1.0, hi=1.0, dtype=np.float32):
    return rng(seed).uniform(lo, hi, size=shape).astype(dtype)


def normal(shape, seed, dtype=np.float32):
    return rng(seed).standard_normal(size=shape).astype(dtype)


def integers(shape, seed, lo, hi):
    """Integers uniform on [lo, hi] inclusive (int64)."""
    return rng(seed).integers(lo, hi + 1, size=shape, dtype=np.int64)


def log_uniform(shape, seed, lo, hi):
    """Positive values with log10 uniform on [log10 lo, log10 hi] (float64)."""
    r = rng(seed).uniform(np.log10(lo), np.log10(hi), size=shape)
    return np.power(10.0, r)


def noise(shape, seed):
    """Standard normal draws (float64) for relative timing noise."""
    return rng(seed).standard_normal(size=shape)


def row_counts(nmodels, seed, lo=40, hi=400):
    """Uneven measurement-set sizes l_k ~ U{lo..hi}."""
    return integers((nmodels,), seed, lo, hi)


def bf16_bits(shape, seed):
    """Random bfloat16 values as uint16 bit patterns: random sign, exponent
    field uniform in [118, 126] (magnitudes 2^-9 .. just under 1), random
    7-bit mantissa."""
    g = rng(seed)
    sign = g.integers(0, 2, size=shape, dtype=np.uint16)
    expo = g.integers(118, 127, size=shape, dtype=np.uint16)
    mant = g.integers(0, 128, size=shape, dtype=np.uint16)
    return (sign << 15) | (expo << 7) | mant
