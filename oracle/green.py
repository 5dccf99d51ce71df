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


def impulse_responses(n, C_ref: np.ndarray, element: str = "q1") -> np.ndarray:
    """Step 1 of Alg. 1: R[alpha, beta, *n] = (K_ref e_{alpha, node 0})_beta."""
    n = tuple(int(k) for k in n)
    d = len(n)
    K_ref = assemble.assemble_K(n, np.ones(n), C_ref, element)
    R = np.zeros((d, d) + n)
    for alpha in range(d):
        imp = np.zeros((d,) + n)
        imp[(alpha,) + (0,) * d] = 1.0
        R[alpha] = assemble.apply(K_ref, imp)
    return R


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


def green_symbol(n, C_ref: np.ndarray, explicit_dft: bool = False, element: str = "q1"):
    """Steps 2-3 of Alg. 1. Returns (K_hat, G_hat), each real [d, d, *n]."""
    n = tuple(int(k) for k in n)
    d = len(n)
    R = impulse_responses(n, C_ref, element)
    axes = tuple(range(2, 2 + d))
    K_c = _transform(R, axes, False, explicit_dft)
    K_hat = 0.5 * (K_c + _reflect(K_c, axes)).real
    blocks = np.moveaxis(K_hat.reshape(d, d, -1), 2, 0)  # [N, d, d]
    G_blocks = np.zeros_like(blocks)
    G_blocks[1:] = np.linalg.inv(blocks[1:])  # frequency 0 is flat index 0
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
    closed form (full Gauss rule), real [d, d, *n]. With t_a = 2 pi k_a / n_a,
    one-minus-cosine written as 2 sin^2(t_a / 2):
      2D: S_a = 2/3 (1 - cos t_a)(2 + cos t_b), K_12 = (lam + mu) sin t_1 sin t_2;
      3D: S_a = 2h/9 (1 - cos t_a) prod_{b != a} (2 + cos t_b),
          K_ab = (lam + mu) h/3 sin t_a sin t_b (2 + cos t_o) (o the third axis);
      K_aa = (lam + 2 mu) S_a + mu sum_{b != a} S_b.
    It equals Alg. 1 (green_symbol) up to rounding but has no cancellation at low
    frequencies, where Alg. 1's transform of O(1) impulse-response entries carries a
    relative error ~eps (n / 2 pi)^2. Used to bracket PCG iteration counts that react
    to that rounding; the solver path itself follows Alg. 1. Square / cubic grids only
    (the formula above is for h equal on every axis)."""
    n = tuple(int(k) for k in n)
    d = len(n)
    if len(set(n)) != 1:
        raise ValueError("closed_form_symbol needs equal axis lengths")
    lam = float(C_ref[0, 1])
    mu = 0.5 * float(C_ref[0, 0] - C_ref[0, 1])
    th = np.meshgrid(*[2 * np.pi * np.arange(k) / k for k in n], indexing="ij")
    c = [np.cos(t) for t in th]
    s = [np.sin(t) for t in th]
    omc = [2.0 * np.sin(0.5 * t) ** 2 for t in th]
    h = 1.0 / n[0]
    K = np.zeros((d, d) + n)
    if d == 2:
        S = [2.0 / 3.0 * omc[0] * (2.0 + c[1]), 2.0 / 3.0 * omc[1] * (2.0 + c[0])]
        K[0, 1] = K[1, 0] = (lam + mu) * s[0] * s[1]
    else:
        S = [2.0 * h / 9.0 * omc[a] * np.prod([2.0 + c[b] for b in range(3) if b != a], axis=0) for a in range(3)]
        for a in range(3):
            for b in range(3):
                if a != b:
                    o = 3 - a - b
                    K[a, b] = (lam + mu) * h / 3.0 * s[a] * s[b] * (2.0 + c[o])
    for a in range(d):
        K[a, a] = (lam + 2.0 * mu) * S[a] + mu * sum(S[b] for b in range(d) if b != a)
    blocks = np.moveaxis(K.reshape(d, d, -1), 2, 0)
    G_blocks = np.zeros_like(blocks)
    G_blocks[1:] = np.linalg.inv(blocks[1:])
    G_hat = np.moveaxis(G_blocks, 0, 2).reshape((d, d) + n)
    return K, G_hat
