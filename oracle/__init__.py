"""CPU oracle for the CASCI sigma build, Davidson-Liu solve and spin-free RDMs.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline / reference leg may import this package; the library under
``paper_2405_10197_gb300`` never does.  The oracle shares no code with the
CUDA path; the two meet only in ``synth_inputs`` (seeded input generators).

Every function is pinned in ``tests/test_oracle_*.py`` against closed forms,
invariants and an independent Fock-space construction of the Hamiltonian.
The mixed-precision error sizes are reported, not asserted: parity unpinned
for that quantity only.
"""
from .driver import (  # noqa: F401
    build,
    strings,
    single_table,
    hij,
    hmat_dense,
    hdiag,
    sigma,
    solve_dense,
    davidson,
    rdm12,
    rdm3,
    rdm2_elements,
    num_threads,
    det_words,
    sci_sigma,
)
from .gas import gas_allowed, sigma_gas, solve_dense_gas  # noqa: F401
from .spin import sector_basis, solve_dense_spin  # noqa: F401
from .aci import aci, aci_epsilon, aci_excluded, aci_reference  # noqa: F401
