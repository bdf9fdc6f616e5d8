"""E4M3 quantisation written from the format's definition, for checking the FP8 search.

E4M3 (the OCP 8-bit floating-point format used by the tensor cores): 1 sign, 4 exponent
(bias 7) and 3 mantissa bits; normal numbers 2^-6 <= |x| <= 448 with spacing 2^(e-3) in the
binade [2^e, 2^(e+1)), subnormals with spacing 2^-9 below 2^-6; no infinities.  Rounding is to
nearest, ties to even, with saturation at 448.  A query row is scaled by the power of two
s = 2^floor(log2(448 / m)), m the row's largest real or imaginary magnitude (float32
arithmetic), s = 1 for a zero row; the atoms are first normalised in float32 by the FP64 norm
and then share one such power of two, from the largest magnitude of the whole dictionary.
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


def normalised_atoms(D: np.ndarray) -> np.ndarray:
    """float32 D_j * (1 / ||D_j||) with the reciprocal of the FP64 norm rounded to float32."""
    D = np.asarray(D, np.complex64)
    n2 = np.sum(np.abs(D.astype(np.complex128)) ** 2, axis=1)
    inv = (1.0 / np.sqrt(n2)).astype(np.float32)
    re = (D.real.astype(np.float32) * inv[:, None]).astype(np.float32)
    im = (D.imag.astype(np.float32) * inv[:, None]).astype(np.float32)
    return re, im


def fp8_scores(Z: np.ndarray, D: np.ndarray, cone: str = "complex") -> np.ndarray:
    """Scores the FP8 search ranks by: |q(D_j)^H q(z)|^2 / (s_z s)^2 (complex cone;
    Re(.) / (s_z s) for the real cone), with the products of quantised values summed exactly
    (float64)."""
    Qz, sz = quantise_rows(Z)
    re, im = normalised_atoms(D)
    m = np.float32(max(np.abs(re).max(), np.abs(im).max()))
    sg = row_scale(np.array([m]))[0]
    Qd = e4m3_round(re.astype(np.float64) * sg) + 1j * e4m3_round(im.astype(np.float64) * sg)
    C = Qz @ Qd.conj().T                       # [n][d] = q(D_j)^H q(z_v)
    if cone == "complex":
        return np.abs(C) ** 2 / (sz[:, None] * sg) ** 2
    return C.real / (sz[:, None] * sg)
