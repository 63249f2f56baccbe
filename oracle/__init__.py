"""FP64 CPU oracle for penalised PET reconstruction by stochastic EM
(Kereta, Twyman, Arridge, Thielemans, Jin: "Stochastic EM methods with
Variance Reduction for Penalised PET Reconstructions").

THIS PACKAGE IS TEST INFRASTRUCTURE.  It is a plain, slow, obviously correct
restatement of what the GPU library computes, used only to check it: only the
tests, the smoke check and the benchmark's CPU-baseline leg may import it.  The
product path (the CUDA library and its Python binding) never imports, calls or
falls back to anything here, and nothing here imports the product path.

Layout of the oracle:
  geometry.py  view angles, bin centres (the parallel-beam geometry)
  siddon.py    explicit sparse system matrix by classical Siddon ray tracing,
               and a brute-force per-pixel line clipper used to pin it
  siddon3d.py  the same for a multi-ring scanner's oblique lines of response
               through a voxel volume, with a per-voxel 3-D clipper
  subsets.py   angle-interleaved ordered-subset partition (§2.1)
  penalty.py   pairwise penalty, potentials of Table 1, parabolic surrogate
               and the closed-form M-step root (§3)
  em.py        likelihood, gradients, subset statistics and the algorithms
               OSEM/MLEM (§2.2), SVREM (§2.3, §3), SAGA and SVRG (§4),
               MAP-EM (the full-batch surrogate EM of §3)

Every image is a float64 array of shape (N, nz) with N = nx*ny pixels in
row-major [iy][ix] order and nz independent slices; every sinogram is
(M, nz) with M = n_angles*n_bins rays in [view][bin] order.  A multi-ring
volume is one column (nx*ny*nz, 1) in [iy][ix][iz] order, its sinogram one
column in [view][bin][ring pair] order.

Parity status of each function is stated in its docstring; the conventions the
paper leaves open (tie-break of rays lying on grid lines, subset sensitivity in
penalised OSEM, the constant SAGA/SVRG preconditioner, step sizes) are marked
"parity unpinned": the oracle and the GPU agree on them by construction only.
"""
