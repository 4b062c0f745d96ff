"""Plain, slow CPU oracle for UniHENN's encrypted CNN inference (arXiv 2402.03060).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import anything here.  The oracle shares no
code, header, table or constant generator with the CUDA library in
``paper_2402_03060_gb300`` and never imports it; the only module both sides use
is ``workloads`` (seeded synthetic inputs, no HE arithmetic).

Parts:
  * ``ckks_ref.c`` / ``ckks.py``  -- RNS-CKKS on CPU (O3): primes, negacyclic NTT,
    FP64 canonical-embedding encoder, keygen, public-key encryption, hybrid key
    switching (ModUp / inner product / ModDown), rotation, relinearisation,
    rescale, decryption.
  * ``layers.py`` -- the paper's layer algorithms (Alg. 1 convolution, Sec. IV-C
    average pooling, Sec. IV-E flatten, Alg. 2 FC, square activation) written
    once against a small backend interface, plus the layout planner (Sec. V).
  * ``slotsim.py`` -- cleartext slot simulator backend (O2): the same layer code
    on FP64 slot vectors with np.roll and masks.
  * ``cnn.py`` -- FP64 plaintext CNN by direct loops (O1).

Parity status: every function is pinned by a ``-m "not gpu"`` test except the
ones listed as "parity unpinned" in their own docstring (none at present).
"""
