"""CPU oracle for the direct n-leg DMRG superblock H·v and its ground-state solvers.

TEST INFRASTRUCTURE ONLY.  Plain, slow, FP64 NumPy/SciPy code written from the
paper (Yamada, Okumura, Machida, arXiv 0707.0159): the Hamiltonian
decomposition of Eq. (dec), the v -> V and v -> V_c reshapes and the three
products H_l V, V H_r^T and H_c V_c.  It shares no code with the CUDA path and
imports nothing from it; the only module both sides use is the seeded input
generator ``paper_0707_0159_gb300.synth``, which holds none of the method's
arithmetic.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
CPU-baseline leg may import this package; the library itself never does.

Modules
-------
columns     exact column operators (spin-1/2 and Hubbard sites, in-column
            Jordan-Wigner strings) for one column of n sites.
superblock  the superblock block 1 · column · column · block 4 and H·v in the
            paper's forms (4-index Eq. (dec), matrix V / V_c forms, explicit
            Kronecker matrix for small sizes, sampled entries).
lattice_ed  brute-force exact diagonalisation of a full n x L ladder in the
            site occupation basis (independent of the superblock code).
solvers     FP64 Lanczos with full reorthogonalisation, Jacobi-Davidson-free
            plain Davidson with the diagonal preconditioner, dense reference.
"""
