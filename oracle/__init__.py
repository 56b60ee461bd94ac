"""FP64 CPU oracle for the pseudo-spectral Navier-Stokes RK4 solver.

This package is TEST INFRASTRUCTURE. It is a plain, slow, obviously correct
restatement of the method of Mortensen & Langtangen, "High performance Python
for direct numerical simulations of turbulent flows" (arXiv 1602.03638):
Sec. 2 (Eqs. NS, realmesh, kmesh, ffteq/iffteq, NSf, mod_pressure, NSfinal,
curl_convection), Sec. 3.1 (wavenumber mesh, Curl/Cross/computeRHS, 2/3-rule
dealiasing) and the Appendix (classical RK4 driver of the Taylor-Green case).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it. The GPU library never imports, links or calls it,
and it shares no code with the GPU library: the only common module is the
seeded input generator, which contains none of the method's arithmetic.

Modules
-------
spectral_ns  -- the solver: transforms, curl, cross product, dealiasing,
                projection, viscous term, RK4, diagnostics.
brute_dft    -- O(N^6) triple-sum DFT used to pin the transform convention.
sgs_mlp      -- FP64 reference of the learned subgrid-stress closure (filter,
                gradients, stress, network forward/backward, closure force).

Parity status of each function is stated in its docstring; the one part with
no independent pin (long-time Taylor-Green Re=1600 statistics, whose workshop
data the paper cites but does not print) says "parity unpinned".
"""

from . import spectral_ns, brute_dft, sgs_mlp  # noqa: F401
