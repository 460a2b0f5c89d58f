"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package holds no arithmetic of the SDRT method.  It only generates
  * structured periodic meshes (element vertices, face adjacency and periodic
    shifts) with the subdivision patterns of the paper's uniform meshes (Sec. 3,
    "mesh patterns": 1 quad/hex, 2 triangles/prisms, 6 tetrahedra per cell), and
  * analytic initial fields evaluated at caller-supplied physical points
    (sine wave, isentropic vortex, Taylor-Green vortex) plus seeded
    perturbations.
"""
