"""Failure detection without a GPU fault: the kernels' bounded waits give up and report
FE_ERR_TIMEOUT through the status word, and the CUDA context stays usable."""
import pytest

import oracle
from paper_1401_3301_gb300 import meshgen
from helpers import check_values, fe_or_skip, to_cuda

pytestmark = pytest.mark.gpu


def test_bounded_wait_runs_out_and_the_context_stays_usable():
    fe = fe_or_skip()
    assert fe.fe_selftest_wait_timeout() == 6  # FE_ERR_TIMEOUT
    m = meshgen.kuhn_cube_mesh(5, seed=90)
    q, me = to_cuda(m.q), to_cuda(m.me)
    p = fe.fe_pattern(q, me)
    vals = fe.fe_assemble_stiff(p, q)
    assert p.status() == (0, -1)
    ref = oracle.assemble(oracle.STIFF, m.q, m.me)
    check_values(vals.cpu().numpy(), ref, 0, "3D stiffness after a bounded wait ran out")
    assert fe.fe_selftest_wait_timeout() == 6  # repeatable
