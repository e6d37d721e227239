"""CPU oracle of the multilevel decomposition (test infrastructure only).

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The GPU library never does.
"""
from .oracle import (  # noqa: F401
    build,
    decompose,
    recompose,
    recompose_classes,
    decompose_adjoint,
    recompose_adjoint,
    line_mass,
    line_prolong,
    line_restrict,
    line_mass_solve,
    uniform_coords,
    max_levels,
    dim_levels,
    decompose_per_dim,
    recompose_per_dim,
    decompose_adjoint_per_dim,
    recompose_adjoint_per_dim,
)
from .quantize import node_classes, quantize, dequantize  # noqa: F401,E402
