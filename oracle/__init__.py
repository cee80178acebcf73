"""Plain FP64 CPU oracle of the FR/LES residual, RK4 update, forces, FW-H
surface sampling and FW-H integration.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports this
package; only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may use it.  It shares no code with the CUDA library: the two
meet only at the seeded mesh/state generators in
``paper_2501_05709_gb300.workloads`` and at the mesh description format.

Everything is written for clarity, vectorised over elements with numpy, in
float64.  Each function cites the passage of the paper (arXiv 2501.05709) it
follows; where the paper is silent (it cites Huynh's FR without giving
points, correction functions, Riemann solver or viscous scheme) the reading
taken is stated in the docstring.
"""
