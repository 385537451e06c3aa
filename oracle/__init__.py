"""FP64 CPU oracle for multiway p-spectral clustering.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import this
package: only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` use it.  It shares no code with the CUDA library; both take
their inputs from ``paper_2605_26975_gb300.workloads``.

Every function is a plain, slow restatement of what the paper defines
("Nonlinear spectral clustering with C++ GraphBLAS", Section 2: Eq. 1, the
p-Laplacian, phi_p and the p-norm; Algorithm 1; Section 3.1: RCut), in float64
with numpy.  Where the paper is silent the module docstrings state the reading
taken.  The pins that tie each function to something other than itself live in
``tests/test_oracle_*.py``.

Parity status: every function is pinned.  The p < 2 stages of the solve, a
continuation with no closed form, are pinned on special cases: the local
quadratic convergence of Newton with the exact Hessian near a smooth
minimiser, and the known global minimum (F_p = 0, RCut = 0) on graphs with k
connected components.  The path through a whole schedule is checked by
agreement of the two implementations.
"""
from .plap import (edge_list, phi_p, abs_pow_pm2, p_norm_p, objective_parts, objective,
                   p_laplacian, euclidean_grad, euclidean_hvp, alg1_sparse_hvp)
from .manifold import (SolveOptions, inner, project, riemannian_hessian, qf, tcg,
                       rtr_newton, solve)
from .cluster import SplitMix64, sq_dist_to, kmeans_pp, lloyd, kmeans, rcut

__all__ = [
    "edge_list", "phi_p", "abs_pow_pm2", "p_norm_p", "objective_parts", "objective",
    "p_laplacian", "euclidean_grad", "euclidean_hvp", "alg1_sparse_hvp",
    "SolveOptions", "inner", "project", "riemannian_hessian", "qf", "tcg", "rtr_newton", "solve",
    "SplitMix64", "sq_dist_to", "kmeans_pp", "lloyd", "kmeans", "rcut",
]
