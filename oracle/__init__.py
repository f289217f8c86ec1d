"""FP64 CPU oracle for the 2-D DWT of Barina et al., "Accelerating Discrete
Wavelet Transforms on GPUs" (arXiv 1705.08266).

THIS PACKAGE IS TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
it. The product path (``paper_1705_08266_gb300``) never imports, links or runs
anything here, and nothing here imports the product path. The two share no
code; only the seeded input generators (``paper_1705_08266_gb300.synth``, which
holds none of the transform's arithmetic) feed both.

Modules
-------
lifting     O1: separable lifting in the paper's step order (Sec. 2, Eq. 2 and
            the separable scheme S_U^V | S_U^H | T_P^V | T_P^H), FP64 for
            CDF 9/7 and linear 5/3; O3: reversible integer LeGall 5/3 in the
            same order; Mallat multilevel recursion on LL.
filterbank  O2: the convolution filter bank G0/G1 followed by subsampling
            (Sec. 2, Eq. 1), with taps derived from the closed-form
            Daubechies half-band factorisation, not from a table.
operators   The paper's 4x4 polyphase lifting matrices (Sec. 2 separable
            T_P^H, T_P^V, S_U^H, S_U^V; Sec. 3 non-separable T_P, S_U and the
            P = P0 + P1 split) turned into explicit matrices acting on small
            images, plus the multiply-accumulate counts of Table 1.

Every function is pinned by ``tests/test_oracle_*.py`` against facts that the
paper and the mathematics fix (lifting == convolution, perfect
reconstruction, vanishing moments, DC gain, Table 1 counts, operator
identities, exhaustive integer round trips). Nothing is pinned against the
CUDA path.
"""
