"""FP64 CPU oracle for certified linearization-error bounds (LEBs) — TEST INFRASTRUCTURE ONLY.

This package is a plain, slow, obviously-correct restatement of what the CUDA path computes,
written from the paper's definitions:

* ``oracle.dynamics``  analytic model equations of App. A (planar quadrotor, spring-coupled chain),
                       their Jacobians (Eq. 8) and hand-derived Hessian entries.
* ``oracle.pbh``       set -> box hull (Eq. 18a, Eq. 21 row-l1 norm), the path-based Hessian bound
                       (Thm. 1, Eq. 15), the expanded and classic interval-Hessian bounds (Eqs. 12-13),
                       and the zonotope map Gamma (Sec. IV-C).
* ``oracle.crown``     MLP forward pass, Jacobian, activation relaxations, CROWN back-substitution
                       (Thm. 2) and the Jacobian-corrected remainder bound (Thm. 3), in torch FP64 on CPU
                       so that its gradient is available for the adjoint checks.
* ``oracle.exact``     exact remainder ranges: 1-D analysis for the planar quadrotor, and
                       activation-pattern enumeration with linear programs for ReLU networks.
* ``oracle.sampling``  sampled true remainders for soundness checks.
* ``oracle.proposer``  the learned bound proposer's MLP forward/backward/Adam step.
* ``oracle.dynamics3d`` the satellite and (coupled) 3-D quadrotor models of App. A with their
                       hand-derived Hessian entries.
* ``oracle.pbh_grad``  the gradient of the PBH bound (differentiable LEBs, Sec. IV-D).
* ``oracle.tube``      the step after the LEB: Ebar_j = [E(z_j) R_j] (Eq. 18b) and the tube centre and
                       width h^mu, h^sigma (Eqs. 20-21) from packed system responses.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import this
package. The product path (``paper_2607_01203_b300``) never imports it, and this package imports
nothing from the product. All arithmetic is FP64 with round-to-nearest (no directed rounding): the
oracle states the bound in exact-real terms up to FP64 rounding, and the CUDA path must contain it
(soundness) while being at most a stated rounding slack wider.

Parity status: every function here is pinned by a ``-m "not gpu"`` test against something other than
itself (closed forms, exact ranges, invariants, brute force). The paper's printed numbers (Tables I-III)
are not reproducible with the published information and pin nothing: "parity unpinned" for those.
"""
