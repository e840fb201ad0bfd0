"""FP64 CPU oracle for the Brownian hard-disk time step -- TEST INFRASTRUCTURE.

This package is a plain, slow, obviously-correct restatement of the method of
Carter, Hitschfeld, Navarro & Soto (arXiv:1703.02484), written from the paper:
Eq. (integration) Euler-Maruyama update (Sec. 2.2), the diffusiophoretic pair
force (Sec. 2.2), the truncated Gaussian noise (Sec. 2.4), the overlap
correction law Eq. (overlaps) iterated as Algorithm 2 with the sigma/4 cap
(Sec. 4.4), the Delaunay triangulation of the disk centres (Sec. 4.1), the
inverted-triangle predicate Eq. (predicate) (Sec. 4.3), the active-Brownian
self-propulsion of Sec. 7, and Verlet neighbour lists (Sec. 5).

Only tests/, __graft_entry__.smoke() and the cpu_baseline / reference legs of
bench.py may import it.  It shares no code with the CUDA library and never
reads anything the CUDA library produced except the state it is asked to step
from.  Every function cites the passage it follows.
"""
from . import philox, noise, forces, dynamics, geometry, periodic, overlap, step, verlet  # noqa: F401
