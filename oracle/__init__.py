"""FP64 CPU oracle for the multicomponent Stefan-Maxwell + compressible (f, g)
lattice Boltzmann step (Sawant, Dorschner & Karlin, arXiv 2004.11286).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` use it.  It shares no code, tables or constants with the
CUDA path; it takes its inputs as plain NumPy arrays.
"""

from .lbm_oracle import (  # noqa: F401
    C, OPP, Q, Params, psi_product, g_ansatz, iso_derivative, stream,
    moments, node_state, sm_momenta, collide, step, run, init_populations,
    macroscopic, collide_patch_center, conserved_sums, Frame, stream_frame, XREF,
)
