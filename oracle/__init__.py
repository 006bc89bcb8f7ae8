"""CPU oracle for the CKKS homomorphic linear transformation.

TEST INFRASTRUCTURE ONLY.  A plain, slow, independent CPU implementation of
what the GPU library computes (RNS-CKKS key switching and the diagonal, BSGS,
DH-BSGS and TH-BSGS linear transformations), written from the paper's
Sec. II-III, Algorithms 1-2 and Eqs. (1)-(8).  Only tests/, the smoke check in
__graft_entry__ and bench.py's CPU-baseline leg may import it; it shares no
code with the GPU library.

Parity pins: every function here is pinned in tests/test_oracle_*.py against
brute force, closed forms or values the paper prints.  Unpinned readings: the
exact construction of the merged ModDown+rescale (pinned only through its
error bound), the key gadget, the prime and root choices (conventions).
"""
