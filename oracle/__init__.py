"""Plain, slow CPU FP64 oracle for the MLMC level batch of Park & Teckentrup,
"Improved Multilevel Monte Carlo Methods for Finite Volume Discretisations of
Darcy Flow in Randomly Layered Media" (arXiv 1506.04694).

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of
``bench.py`` may import it.  The product path (``paper_1506_04694_gb300``)
never imports, links or executes anything in here, and nothing in here
imports the product path.

Every function follows the paper's definitions in its own order and notation,
in numpy/scipy FP64; library primitives (``numpy.fft.fft2``,
``scipy.linalg.solveh_banded``, ``math.fsum``) serve as single steps only.

Modules
-------
philox  -- counter-based Philox4x64-10 words, uniforms, Box-Muller normals
darcy   -- random layers, circulant-embedding fields (Ex. 1, Ex. 2, Eq. 2.3),
           cell-centred TPFA assembly with harmonic faces (Sec. 3.1, Eq. 3.3),
           direct banded solve, outflow QoI M^(2) (Sec. 3.4)
mlmc    -- level batch with plain and Coarse Grid Variates coupling
           (Eq. 3.6, Eq. 4.1, Eq. 4.2), exactly rounded level sums, sample
           sizes from the even eps^2 split (Eq. 3.7) and the MLMC estimate

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, library routines, brute force or exact moments; none
is "parity unpinned".
"""
from . import philox, darcy, mlmc  # noqa: F401
from .darcy import Model  # noqa: F401
