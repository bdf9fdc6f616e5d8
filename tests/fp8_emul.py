"""E4M3 quantisation written from the format's definition, for checking the FP8 search.

E4M3 (the OCP 8-bit floating-point format used by the tensor cores): 1 sign, 4 exponent
(bias 7) and 3 mantissa bits; normal numbers 2^-6 <= |x| <= 448 with spacing 2^(e-3) in the
binade [2^e, 2^(e+1)), subnormals with spacing 2^-9 below 2^-6; no infinities.  Rounding is to
nearest, ties to even, with saturation at 448.  Rows are scaled by the power of two
s = 2^floor(log2(448 / m)), m the row's largest real or imaginary magnitude (float32
arithmetic), s = 1 for a zero row.
"""
import numpy as np


def e4m3_round(x: np.ndarray) -> np.ndarray:
    x = np.asarray(x, np.float64)
    a = np.abs(x)
    e = np.floor(np.log2(np.where(a > 0, a, 1.0)))
    e = np.maximum(e, -6.0)            # subnormal range shares the spacing of the 2^-6 binade
    ulp = np.exp2(e - 3.0)
    q = np.round(a / ulp) * ulp        # numpy rounds halves to even
    q = np.minimum(q, 448.0)
    return np.sign(x) * q


def row_scale(m: np.ndarray) -> np.ndarray:
    m = np.asarray(m, np.float32)
    out = np.ones(m.shape, np.float64)
    ok = (m > 0) & np.isfinite(m)
    r = np.float32(448.0) / m[ok]
    _, ex = np.frexp(r)                 # r = f 2^ex with f in [0.5, 1): floor(log2 r) = ex - 1
    out[ok] = np.exp2(np.clip(ex - 1, -126, 126).astype(np.float64))
    return out


def quantise_rows(V: np.ndarray):
    """(quantised complex128 rows in scaled units, scale per row) of complex64 rows V."""
    V = np.asarray(V, np.complex64)
    m = np.maximum(np.abs(V.real), np.abs(V.imag)).max(axis=1)
    s = row_scale(m)
    Vs = V.astype(np.complex128) * s[:, None]
    return e4m3_round(Vs.real) + 1j * e4m3_round(Vs.imag), s


def fp8_scores(Z: np.ndarray, D: np.ndarray, cone: str = "complex") -> np.ndarray:
    """Scores the FP8 search ranks by: |q(D_j)^H q(z)|^2 / (s_z^2 s_j^2 ||D_j||^2) (complex
    cone; Re(.) / (s_z s_j ||D_j||) for the real cone), with the products of quantised values
    summed exactly (float64)."""
    Qz, sz = quantise_rows(Z)
    Qd, sd = quantise_rows(D)
    n2 = np.sum(np.abs(np.asarray(D, np.complex128)) ** 2, axis=1)
    C = Qz @ Qd.conj().T                       # [n][d] = q(D_j)^H q(z_v)
    if cone == "complex":
        return np.abs(C) ** 2 / (sz[:, None] ** 2 * (sd ** 2 * n2)[None, :])
    return C.real / (sz[:, None] * (sd * np.sqrt(n2))[None, :])
