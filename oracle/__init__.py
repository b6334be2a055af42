"""Oracle for sign(H_W(mu)) b — TEST INFRASTRUCTURE ONLY.

A plain, slow, FP64 CPU restatement of what the hot path computes, written from the
paper (Bloch et al., "Short-recurrence Krylov subspace methods for the overlap Dirac
operator at nonzero chemical potential", arXiv:0910.1048). Only the test suite,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs of
``bench.py`` may import it. The CUDA library never imports, links or runs it, and it
shares no code with the CUDA library; the only common module is ``synth`` (seeded
input generators).

Modules
  gamma      Euclidean chiral gamma matrices
  wilson     dense and matrix-free D_W(mu), H_W(mu) = gamma5 D_W(mu)
  matsign    sign(A) by eigendecomposition (Eq. 1), scaled Roberts-Newton, eigh
  freefield  closed-form sign(H_W) for unit links, any lattice size
  rational   Neuberger/Kenney-Laub g_s (Eqs. neuberger_mit_c, pfe_s), Theorem 1,
             pole count (Eq. no_of_poles), Zolotarev coefficients
  lanczos    direct two-sided Lanczos-LR (Algorithm 4) and multishift iterates
             V_k (T_k - sigma_i)^-1 e1 (Section 2.2, Algorithm 3)
  deflation  critical eigenpairs, x_P (Eq. exact_proj), r, modified shadow vector
  fom        restarted FOM-LR(m, k) with a rational function, Algorithm 1 (Arnoldi by modified
             Gram-Schmidt, one basis for all shifts, restarts through the collinear residuals)
  krylov     plain C (OpenMP) FP64 matrix-free H_W(mu) and two-sided Lanczos, Algorithm 4 at
             any lattice size (krylov.c, compiled with gcc on first use or by build_lib())

Parity status: every function is pinned by a "not gpu" test against closed forms,
invariants, brute force or a library routine, except where a module header says
"parity unpinned".
"""
