"""The paper's own parameter shapes (Table "HE parameters"): Set-A dense at full
size (N = 2^13, L+1 = 5, alpha = 5, beta = 1, n = 4096 diagonals, split
(2^4)^3), and Set-B's parameters (N = 2^15, L+1 = 16, alpha = 8, beta = 2,
k = 8) with 256 diagonals; output residues bit-exact with the oracle.

Both sets use 54-bit words, so the input and the diagonals are encoded at
2^47: the rescale by a 54-bit prime then leaves the output at 2^40, the same
output scale as the 40-bit-prime workloads.  At 2^40 x 2^40 the output would
sit at 2^26, and the fast basis conversion of the merged ModDown and rescale
(Eq. 4 over {q_last} and the k special primes) leaves an integer error of up to
k + 1 in each coefficient of c1 -- about 0.17 in the slots at that scale for
Set-B (0.02 with a single diagonal, where only q_last's limb is nonzero)."""
import numpy as np
import pytest

from oracle import lt as olt
from oracle.workload import add_keys, make_problem

from gpu_common import assert_same, gpu_context, upload_problem

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,D,split", [("setA", 4096, (16, 16, 16)), ("setB", 256, (4, 8, 8))])
def test_paper_parameter_sets(name, D, split):
    pb = make_problem(name, 21, D, log_scale=47, log_diag_scale=47)
    add_keys(pb, olt.rotation_set("th", D, split, 1, pb.ctx.N // 2))
    g = gpu_context(name)
    f = upload_problem(g, pb)
    out, _ = g.lt_eval(g.ct_from_host(np.stack(pb.ct)), f, "th", split)
    got = out.numpy()
    assert_same(got, np.stack(olt.lt_th_bsgs(pb.ctx, pb.ct, pb.diags, pb.keys, *split)[0]), name)
    y = pb.decrypt((got[0], got[1]))
    e = y - pb.expected()
    assert float(np.max(np.maximum(np.abs(e.real), np.abs(e.imag)))) <= 1e-4
