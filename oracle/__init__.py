"""FP64 CPU oracle for the tensor-train discrete-ordinates (TT-S_N) time step.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA path and never imports it.

Modules (each function cites the passage of arXiv 2503.18056 it follows):

* ``angles``   -- latitude-longitude angular grid (Sec. 3).
* ``quartic``  -- the per-cell quartic for the intermediate temperature
                  (Sec. 3.2, Eq. couple_b), by bisection.
* ``dense``    -- plain dense S_N stepper: upwind finite-volume transport
                  (Sec. 3.1, Eq. lhs / Eq. upwind) and the backward-Euler
                  source with the energy-conserving temperature update
                  (Sec. 3.2).
* ``tt``       -- tensor-train arithmetic of Sec. 4.1 (addition, Hadamard
                  product, integration) plus expansion to the full tensor.
* ``rounding`` -- Algorithm 1 with the TT-SVD truncation (App. A.1) and with
                  the Gram-SVD truncation (App. A.2, Eq. gramfinal).
* ``ttstep``   -- the step-then-truncate TT stepper of Sec. 4.3-4.5 on the
                  paper's grouped-space three-core layout (Eq. tensor_decomp).
* ``split``    -- the same step on the split-space layout (one core per
                  spatial axis, then theta and phi; Sec. 4.1, Sec. 7), with
                  the spatial fields s and e entering as TT-SVDs of the field.
* ``adjoint``  -- the escape-energy gradient (reverse sweep of the dense step).
* ``analytic`` -- analytic solutions of the validation problems of Sec. 5
                  (hohlraum mean intensity, Gaussian line source).

Every function here is pinned by ``-m "not gpu"`` tests against closed forms,
invariants and brute force; none is "parity unpinned".
"""
