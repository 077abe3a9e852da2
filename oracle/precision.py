"""Reduced-precision storage of the quasi-1D factors (the precision pattern).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The sweep applies each stored T_i = S_i^{-1} to a vector; the setup computes
T_i in full precision and only its stored copy is rounded.  Two stored forms
besides plain FP32, both with one power-of-two scale per block:

  * fp16        T_i = 2^e q,          q = fp16(T_i / 2^e)
  * split_fp16  T_i = 2^e (hi + lo),  hi = fp16(T_i / 2^e),
                                      lo = fp16(T_i / 2^e - hi)

real and imaginary parts rounded separately (round to nearest even).  The
exponent puts the largest scaled component just below 2^15 (fp16's largest
finite value is 65504), so no entry overflows and every entry above
2^-14 in scaled units (2^-29 of the block's largest) keeps fp16's full
11-bit significand.  Rounding errors per scaled component z:
  fp16:        |fp16(z) - z|        <= 2^-11 |z|            (|z| >= 2^-14)
  split_fp16:  |hi + lo - z|        <= 2^-22 |z| + 2^-25
(hi carries z to 2^-11 |z|; lo carries the remainder, itself rounded to 2^-11
of its size, or to half fp16's smallest subnormal 2^-24 when the remainder
lies in the subnormal range).  The precision pattern then runs the outer
Krylov iteration on the FP64 true residual, so the solution accuracy is set
by the tolerance, not by the stored precision.
"""
from __future__ import annotations

import math

import numpy as np

FORMATS = ("fp32", "fp16", "split_fp16")
SCALE_TOP = 15          # largest scaled component lies in [2^14, 2^15)


def block_exponent(T: np.ndarray) -> int:
    """e with max(|Re T|, |Im T|) / 2^e in [2^14, 2^15); 0 for a zero block."""
    mx = float(max(np.max(np.abs(T.real)), np.max(np.abs(T.imag))))
    if mx == 0.0:
        return 0
    _, ex = math.frexp(mx)          # mx = f 2^ex, f in [0.5, 1)
    return ex - SCALE_TOP


def _fp16(x: np.ndarray) -> np.ndarray:
    return x.astype(np.float16).astype(np.float64)


def fp16_parts(T: np.ndarray):
    """(q, e): q complex with fp16-exact parts, T ~= 2^e q."""
    e = block_exponent(T)
    z = T / 2.0 ** e
    return _fp16(z.real) + 1j * _fp16(z.imag), e


def split_fp16_parts(T: np.ndarray):
    """(hi, lo, e): T ~= 2^e (hi + lo), hi and lo with fp16-exact parts."""
    e = block_exponent(T)
    z = T / 2.0 ** e
    hr, hi_ = _fp16(z.real), _fp16(z.imag)
    lr, li = _fp16(z.real - hr), _fp16(z.imag - hi_)
    return hr + 1j * hi_, lr + 1j * li, e


def round_factor(T: np.ndarray, fmt: str) -> np.ndarray:
    """The value the sweep uses for a stored block T in format fmt (FP64 result)."""
    if fmt == "fp32":
        return T.real.astype(np.float32).astype(np.float64) + 1j * T.imag.astype(np.float32).astype(np.float64)
    if fmt == "fp16":
        q, e = fp16_parts(T)
        return q * 2.0 ** e
    if fmt == "split_fp16":
        hi, lo, e = split_fp16_parts(T)
        return (hi + lo) * 2.0 ** e
    raise ValueError("unknown factor format %r" % (fmt,))
