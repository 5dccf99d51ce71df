"""FP64 CPU oracle for the J-FFT solver (Ladecky et al., arXiv 2508.02613).

TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT. Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs of
``bench.py`` may import this package. The CUDA library never calls it, and it
never calls the CUDA library: the two share no code. Only the seeded input
generators in ``synthetic/`` feed both.

What it computes, step by step in the paper's notation, in plain NumPy/SciPy:
  * ``fe``        Q1 element (bilinear quad / trilinear hex, full 2^d Gauss rule),
                  Mandel B matrices and isotropic C (Sec. 2.1, Sec. 4 "Constitutive law");
  * ``assemble``  sparse K = B^T W C B and f = -B^T W C E by element-wise
                  assembly on the periodic grid (Eq. lin_system_exp);
  * ``green``     Alg. 1: impulse responses of K_ref, component-wise DFT, d x d
                  inversion with the zero frequency pinned to 0 (Eq. prec_lin_systemG_FFT);
  * ``jacobi``    diag(K) from the assembled matrix and by Alg. 2 (impulse combs),
                  the void rule, and J^(1/2) (Sec. 3.2, Eq. Jacobi);
  * ``pcg``       textbook PCG (Saad, Alg. 9.1), x_0 = 0 (Sec. 4 "Initial solution");
  * ``post``      zero-mean fluctuation, element-averaged stress, homogenised
                  stiffness (Eq. aim_fun, Sec. 5.3);
  * ``dense``     brute-force dense pseudo-inverse solve for tiny grids;
  * ``material``  E = E_min + (E_max - E_min) rho^p per voxel.

Pins (checked by ``tests/test_oracle_*.py``, run with ``-m "not gpu"``): textbook
Q1 element entries, symmetry / semidefiniteness / rigid-translation kernel of K,
Alg. 1 equal to a hand-derived closed-form symbol and to an explicit DFT, Alg. 2
equal to the assembled diagonal, one-iteration convergence on homogeneous
material, dense brute force, the laminate closed form, Hill bounds, the energy
identity, element stresses against a nodal-difference brute force and against the
laminate's constant normal stress, the node-by-node operator against the assembled
one, and the paper's printed material constants. Exact PCG iteration counts at the benchmark
workloads have no printed value in the paper: parity unpinned for those counts
(they are compared GPU-vs-oracle only).
"""
