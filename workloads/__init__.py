"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This package holds mesh topology, coordinates, boundary sets, the partition
of elements into subdomains, the analytic fibre specification and the load
schedule, and nothing of the method's arithmetic: no shape functions, no
quadrature, no constitutive law, no solver step.  Both the oracle and the
library read these dictionaries; neither shares any other code.

Conventions (they are part of the library's public input format):

* Hexahedra (Q1: 8 nodes, Q2: 27 nodes) use lexicographic local numbering:
  local node ``a + (k+1)*(b + (k+1)*c)`` sits at reference point
  ``(-1 + 2a/k, -1 + 2b/k, -1 + 2c/k)`` for ``a, b, c in 0..k``.
* Local faces of a hexahedron: 0 = xi-, 1 = xi+, 2 = eta-, 3 = eta+,
  4 = zeta-, 5 = zeta+.
* Degrees of freedom are interleaved per node (x, y, z), Section 4 of the
  paper; a Dirichlet node has all three components clamped.
"""
from .slab import slab_problem, slab_config, SLAB_CONFIGS, box_groups  # noqa: F401
from .lv import lv_problem, lv_config, lv_part_problem, clamped_parts, LV_CONFIGS  # noqa: F401
from .material import default_material  # noqa: F401
