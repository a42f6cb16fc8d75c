"""CPU FP64 oracle for the decentralized major/minor-cycle imaging path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
its Python binding) imports, calls or links anything here; only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline legs of ``bench.py`` do.

Every function is a plain, slow, obviously-correct restatement of the
arithmetic it names, in float64, following arXiv 2507.22128
("A Decentralized Framework for Radio-Interferometric Image Reconstruction"):

* ``dft``        direct measurement operator of Eq. 1 (C = D = 1) and its
                 adjoint (dirty image, PSF, Eq. 2 residual)
* ``es``         exponential-of-semicircle kernel and its Fourier transform
* ``gridder``    w-stacked ES gridding / degridding (G, G^dagger of Eq. 2)
* ``partition``  |uv| partitioning into overlapping domains (Sec. 3) and the
                 tile sort order of the samples
* ``filters``    Fourier-domain filters Gamma_p and padded convolutions
* ``wavelet``    Daubechies-4 filter from its spectral factorisation and the
                 periodic orthonormal 2D DWT
* ``fista``      Eq. 4 / Eq. 5 minor cycle
* ``msclean``    Eq. 6 / Eq. 7 minor cycle
* ``framework``  the decentralized loop: fill, rho aggregate, exchange,
                 image update (Eq. 3) and the final combine

The oracle shares no code with the CUDA path.  Both consume the seeded
synthetic inputs of ``paper_2507_22128_gb300.synth`` (inputs only).

Parity status of each function is stated in its module docstring; every
function here is pinned by a ``-m "not gpu"`` test in ``tests/test_oracle_*``.
"""
