"""Green preconditioner M^-1 = F^-1 G_hat F (paper Sec. 3.1, Eq. prec_lin_systemG_FFT, Alg. 1).

Alg. 1, as read here:
  Step 1: for each component alpha, apply K_ref (uniform reference material) to a
          unit impulse in component alpha at node 0; the response is row alpha of
          the impulse-response array R[alpha, beta, N_1..N_d].
  Step 2: component-wise DFT of every R[alpha, beta]. (The printed loop range
          "{0..d}^d" and the in-place transform of K_hat are read as (alpha, beta)
          in {1..d}^2 and K_hat[alpha, beta] = F(R[alpha, beta]).)
  Step 3: invert the d x d block at every frequency; the zero frequency block is
          set to 0 (zero-mean constraint; the printed index [:, :, 1, 1, 1] is read
          as "the zero frequency" for any d).

DFT convention (unstated in the paper): unnormalised forward transform
F[k] = sum_I x[I] exp(-2 pi i k.I / n), inverse with 1/N, i.e. numpy.fft.fftn /
ifftn. With this convention (K u)_beta = F^-1( sum_alpha K_hat[alpha, beta] F(u_alpha) ),
so the block acting on the vector of transformed components is K_hat^T; the
oracle applies exactly that transpose (for the centrosymmetric Q1 stencil K_hat is
real symmetric, so the transpose is immaterial, which a test asserts).

Real, even symbol. The impulse response of the uniform reference operator is even
in the node offset (the Q1 stencil is centrosymmetric), so its transform is the
cosine sum K_hat(k) = sum_I R(I) cos(2 pi k.I / n): real, and equal at k and -k.
A complex FFT of R returns that only up to rounding; the rounding-level imaginary
and odd parts make F^-1 G_hat F slightly non-symmetric, and PCG with the
Green-Jacobi preconditioner is sensitive to that (its iteration counts move by
several at 256 x 256 and above). Step 2 therefore keeps the real part of the mean
of the transform at k and at -k, which is the cosine sum above evaluated with the
FFT, and the symbol is returned real.
"""

from __future__ import annotations

import numpy as np

from . import assemble


def impulse_responses(n, C_ref: np.ndarray, element: str = "q1", dtype=np.float64) -> np.ndarray:
    """Step 1 of Alg. 1: R[alpha, beta, *n] = (K_ref e_{alpha, node 0})_beta, K_ref the
    operator of the uniform reference material, applied matrix-free (in ``dtype``)."""
    n = tuple(int(k) for k in n)
    d = len(n)
    R = np.zeros((d, d) + n, dtype=dtype)
    for alpha in range(d):
        imp = np.zeros((d,) + n, dtype=dtype)
        imp[(alpha,) + (0,) * d] = 1
        R[alpha] = assemble.apply_matrix_free(n, np.ones(n, dtype=dtype), np.asarray(C_ref).astype(dtype), imp,
                                              element)
    return R


def block_inverse(blocks: np.ndarray) -> np.ndarray:
    """Inverse of every d x d block of [m, d, d] (d = 2, 3) by the adjugate formula, in the
    blocks' own floating-point type (numpy.linalg has no extended-precision inverse)."""
    d = blocks.shape[-1]
    K = blocks
    if d == 2:
        det = K[:, 0, 0] * K[:, 1, 1] - K[:, 0, 1] * K[:, 1, 0]
        adj = np.stack([np.stack([K[:, 1, 1], -K[:, 0, 1]], -1), np.stack([-K[:, 1, 0], K[:, 0, 0]], -1)], -2)
    elif d == 3:
        c = lambda i, j, k, l: K[:, i, k] * K[:, j, l] - K[:, i, l] * K[:, j, k]  # noqa: E731
        adj = np.stack([np.stack([c(1, 2, 1, 2), -c(0, 2, 1, 2), c(0, 1, 1, 2)], -1),
                        np.stack([-c(1, 2, 0, 2), c(0, 2, 0, 2), -c(0, 1, 0, 2)], -1),
                        np.stack([c(1, 2, 0, 1), -c(0, 2, 0, 1), c(0, 1, 0, 1)], -1)], -2)
        det = K[:, 0, 0] * adj[:, 0, 0] + K[:, 0, 1] * adj[:, 1, 0] + K[:, 0, 2] * adj[:, 2, 0]
    else:
        raise ValueError("d must be 2 or 3")
    return adj / det[:, None, None]


def dft(x: np.ndarray, axes, inverse: bool = False) -> np.ndarray:
    """Explicit O(N^2) multidimensional DFT by dense matrices along each axis (small grids)."""
    y = np.asarray(x, dtype=np.complex128)
    for ax in axes:
        m = y.shape[ax]
        j = np.arange(m)
        sign = 1.0 if inverse else -1.0
        W = np.exp(sign * 2j * np.pi * np.outer(j, j) / m)
        if inverse:
            W = W / m
        y = np.moveaxis(np.tensordot(W, np.moveaxis(y, ax, 0), axes=(1, 0)), 0, ax)
    return y


def _transform(x, axes, inverse, explicit):
    if explicit:
        return dft(x, axes, inverse)
    return np.fft.ifftn(x, axes=axes) if inverse else np.fft.fftn(x, axes=axes)


def _reflect(x: np.ndarray, axes) -> np.ndarray:
    """x evaluated at -k on the periodic frequency grid (index k -> (n - k) mod n)."""
    return np.roll(np.flip(x, axes), 1, axes)


def support_transform(R: np.ndarray) -> np.ndarray:
    """Step 2 of Alg. 1 evaluated over the support of the impulse responses.

    R[alpha, beta, *n] is nonzero only at the few nodes that share an element with
    node 0, and each R[alpha, beta] sums to zero over the grid (K_ref maps a rigid
    translation to zero, Sec. 2). With the DFT convention above its transform is the
    cosine sum, and subtracting the zero sum times 1 turns each cos into cos - 1 =
    -2 sin^2:
        K_hat(k) = sum_J R(J) cos(2 pi k.J / n) = -2 sum_J R(J) sin^2(pi k.J / n).
    Every term is then computed to a few ulps, where the FFT's cosine sum loses
    relative accuracy ~eps (n / 2 pi)^2 at the lowest frequencies. J is taken in the
    symmetric range (-n/2, n/2] (sin^2(pi k.J/n) has period n in J), k over the full
    frequency grid, and the phase k.J/n is reduced to [-1/2, 1/2] before the sine; the
    result is real and even in k by construction."""
    d = R.ndim - 2
    n = R.shape[2:]
    K = np.zeros(R.shape, dtype=R.dtype)
    pi = np.arccos(np.asarray(-1, dtype=R.dtype))   # pi in the responses' precision
    ks = np.meshgrid(*[np.arange(m, dtype=R.dtype) for m in n], indexing="ij")
    support = np.argwhere(np.any(R.reshape((-1,) + n) != 0.0, axis=0))
    for J in support:
        Js = [int(j) if j <= m // 2 else int(j) - m for j, m in zip(J, n)]
        phase = sum(ks[a] * (Js[a] / np.asarray(n[a], dtype=R.dtype)) for a in range(d))  # exact: dyadic
        phase = phase - np.round(phase)   # exact; sin^2(pi x) has period 1 in x, and
        s2 = np.sin(pi * phase) ** 2      # |x| <= 1/2 keeps pi x free of cancellation
        for a in range(d):
            for b in range(d):
                r = R[(a, b) + tuple(J)]
                if r != 0.0:
                    K[a, b] += -2.0 * r * s2
    return K


def green_symbol(n, C_ref: np.ndarray, explicit_dft: bool = False, element: str = "q1",
                 transform: str = "support", dtype=np.float64):
    """Steps 2-3 of Alg. 1. Returns (K_hat, G_hat), each real [d, d, *n].

    ``transform="support"`` (default) evaluates step 2 as ``support_transform``;
    ``transform="fft"`` takes the full transform of R (numpy.fft, or the explicit
    O(N^2) DFT with ``explicit_dft``) and keeps the real part of the mean at k and -k
    (the real, even symbol); the two agree to the FFT's rounding. Step 3 inverts each
    block by its adjugate. ``dtype`` (support form only): the floating-point type of
    the whole computation (numpy.longdouble for the extended-precision oracle)."""
    n = tuple(int(k) for k in n)
    d = len(n)
    if dtype != np.float64 and (transform != "support" or explicit_dft):
        raise ValueError("extended precision is available for the support form only")
    R = impulse_responses(n, C_ref, element, dtype)
    axes = tuple(range(2, 2 + d))
    if transform == "support" and not explicit_dft:
        K_hat = support_transform(R)
    elif transform in ("fft", "support"):
        K_c = _transform(R, axes, False, explicit_dft)
        K_hat = 0.5 * (K_c + _reflect(K_c, axes)).real
    else:
        raise ValueError(transform)
    blocks = np.moveaxis(K_hat.reshape(d, d, -1), 2, 0)  # [N, d, d]
    G_blocks = np.zeros_like(blocks)
    G_blocks[1:] = block_inverse(blocks[1:])  # frequency 0 is flat index 0
    G_hat = np.moveaxis(G_blocks, 0, 2).reshape((d, d) + n)
    return K_hat, G_hat


def apply_green(G_hat: np.ndarray, r: np.ndarray, explicit_dft: bool = False) -> np.ndarray:
    """z = F^-1 G_hat F r for r of shape [d, *n] (the transpose reading above)."""
    d = r.shape[0]
    axes = tuple(range(1, 1 + d))
    r_hat = _transform(r, axes, False, explicit_dft)
    z_hat = np.einsum("ab...,a...->b...", G_hat, r_hat)
    return _transform(z_hat, axes, True, explicit_dft).real


def apply_green_jacobi(G_hat: np.ndarray, J_half: np.ndarray, r: np.ndarray) -> np.ndarray:
    """z = J^(1/2) F^-1 G_hat F J^(1/2) r (paper Eq. prec_lin_systemJG_2)."""
    return J_half * apply_green(G_hat, J_half * r)


def closed_form_symbol(n, C_ref: np.ndarray):
    """(K_hat, G_hat) of the uniform Q1 operator for an isotropic C_ref from the plane-wave
    closed form (full Gauss rule), real [d, d, *n], on a grid with element sides
    h_a = 1 / n_a. With t_a = 2 pi k_a / n_a and V = prod_a h_a, the Q1 stencil factors
    into 1D stiffness 2 (1 - cos t) / h^2, 1D mass (2 + cos t) / 3 and 1D gradient
    i sin t / h per axis:
      S_a    = V / h_a^2 * 2 (1 - cos t_a) * prod_{b != a} (2 + cos t_b) / 3,
      T_ab   = V / (h_a h_b) * sin t_a sin t_b * prod_{o != a, b} (2 + cos t_o) / 3,
      K_aa   = (lam + 2 mu) S_a + mu sum_{b != a} S_b,   K_ab = (lam + mu) T_ab,
    with 1 - cos t written as 2 sin^2(t / 2) and t taken in (-pi, pi]. It equals Alg. 1
    (green_symbol) in exact arithmetic but is computed from the element's formulas
    alone: no impulse response, so no cancellation of large stencil entries."""
    n = tuple(int(k) for k in n)
    d = len(n)
    lam = float(C_ref[0, 1])
    mu = 0.5 * float(C_ref[0, 0] - C_ref[0, 1])
    h = [1.0 / k for k in n]
    V = float(np.prod(h))
    # signed frequencies k in (-n/2, n/2]: the same angles mod 2 pi, and |theta| <= pi
    # keeps sin(theta / 2) free of the cancellation near theta = 2 pi
    th = np.meshgrid(*[2 * np.pi * np.fft.fftfreq(k, 1.0 / k) / k for k in n], indexing="ij")
    c = [np.cos(t) for t in th]
    s = [np.sin(t) for t in th]
    omc = [2.0 * np.sin(0.5 * t) ** 2 for t in th]
    mass = [(2.0 + ci) / 3.0 for ci in c]
    K = np.zeros((d, d) + n)
    S = []
    for a in range(d):
        Sa = V / h[a] ** 2 * 2.0 * omc[a]
        for b in range(d):
            if b != a:
                Sa = Sa * mass[b]
        S.append(Sa)
    for a in range(d):
        for b in range(d):
            if a != b:
                T = V / (h[a] * h[b]) * s[a] * s[b]
                for o in range(d):
                    if o not in (a, b):
                        T = T * mass[o]
                K[a, b] = (lam + mu) * T
        K[a, a] = (lam + 2.0 * mu) * S[a] + mu * sum(S[b] for b in range(d) if b != a)
    blocks = np.moveaxis(K.reshape(d, d, -1), 2, 0)
    G_blocks = np.zeros_like(blocks)
    G_blocks[1:] = block_inverse(blocks[1:])
    G_hat = np.moveaxis(G_blocks, 0, 2).reshape((d, d) + n)
    return K, G_hat
