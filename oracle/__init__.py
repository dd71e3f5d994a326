"""Serial FP64 CPU oracle of the MTPT time step (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its binding) never imports, links or executes anything here, and nothing here
imports the product package.

The arithmetic lives in ``mtpt_oracle.c`` (plain C, ``-O2 -ffp-contract=off``,
no fast-math); ``oracle.py`` is a ctypes binding over numpy arrays and
``analytic.py`` holds the closed-form solutions used as pins.

Parity status of each oracle function (what pins it to something other than
itself; the tests named are under ``tests/``):

* ``philox4x32_10``     -- pinned by test_oracle_rng.py word for word to a
  third-party implementation of the same published generator (PyTorch's
  host-side Philox engine, called as a library routine) over random and
  edge-case counters and keys, plus avalanche and uniformity statistics.
* ``box_muller``        -- pinned to the float64 Box-Muller formula on the
  same words (which word gives the radius, which the angle, and the uniform
  map), and ``normals`` to ``box_muller`` of the library's words.
* ``log_f32``, ``sincos_2pi_f32`` -- pinned to numpy's float64 log/sin/cos
  over every input the walk can produce (error bounds in ulps).
* ``normals``           -- pinned by a Kolmogorov-Smirnov test against N(0,1)
  and by the first four moments.
* ``random_walk``       -- pinned by displacement variance 2 D_RW dt, zero
  mean, walls never crossed, exact mirror images at the walls.
* ``pairs``             -- brute force pinned to hand-built lattices whose
  neighbour sets are known by construction (inclusive cutoff, exact ties);
  the K-D tree pinned to brute force.
* ``mass_transfer``     -- pinned to the two-particle closed form
  W_12 = e / (1 + e), a three-particle hand case, bit-exact invariance of
  uniform masses, exact conservation up to rounding, the maximum principle,
  and the erf solution of the diffusion equation (Sec. 2.1) at the paper's
  density.
* ``run``               -- pinned to the erf solution (pure random walk,
  pure mass transfer and the 50/50 split) and to the spreading of a Gaussian
  point source (variance grows by 2 D t per axis).
* ``react``             -- (bimolecular reaction A + B -> 0, the reading of
  the extension named in Sec. 8) pinned to the closed-form solution of the
  rate law in 50-digit arithmetic (both species, the one in deficit to its
  relative precision), to the composition of substeps, and to a stiff ODE
  integrator; ``particle_rate`` to k N / V.
* ``run_reactive``      -- pinned to plain ``run`` of each species when
  k = 0 (bit for bit), to the well-mixed solution for uniform species, to
  the conservation of sum(M_A - M_B) and to positivity.
"""
from .oracle import *  # noqa: F401,F403
from . import analytic  # noqa: F401
