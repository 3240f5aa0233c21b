"""Plain FP64 CPU oracle for the LiveCap Gauss-Newton hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports, links or runs
this package.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may use it.  It shares no code with the CUDA
path; the only thing both consume is the seeded scene generator in ``synth``.

Modules
-------
graph       farthest-point node sampling, K-nearest-node binding with
            (1 - d/d_max)^2 weights, node edges and material edge weights.
nonrigid    embedded-graph warp, pinhole projection, bilinear image and
            gradient sampling, photometric / silhouette / ARAP residuals, the
            assembled sparse Jacobian, Jacobi-PCG on J^T J, Gauss-Newton and
            the energy (Sec. 3.4 and Sec. 4 of the paper), in FP64.
visibility  the integer / FP32-exact decisions: z-buffer visibility, the
            contour set B and the silhouette directions b_i.  Written in plain
            C (``visibility.c``) so that its FP32 operations are the specified
            ones; this is the one place the oracle is not FP64, because the
            decisions must be taken in the kernel's precision.
pose        the skeletal stage-1 fit (Sec. 3.3): forward kinematics, linear
            blend skinning, 2D / 3D joint and silhouette residuals, dense
            normal equations solved by a Cholesky factorisation.
surface     the paper's own per-vertex formulation of the non-rigid stage
            (unknowns V; E_smooth, E_edge, E_velocity, E_acceleration beside
            the data terms), its sparse Jacobian and Gauss-Newton, in FP64.
dt          the silhouette distance transform (exact squared distances to
            the contour pixels, FP32 square root).
mlp         the learned per-node warm start network in FP64 (forward,
            backward, Adam), the reference for the BF16 kernels.
"""
