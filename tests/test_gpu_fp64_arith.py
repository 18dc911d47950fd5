"""The contracted FP64 form's own square root and reciprocal (the hardware's
approximate seed refined by one third-order step: Householder's iteration
for the square root, the cubic Newton-Raphson step for the reciprocal) stay
within one ulp of the correctly rounded results of CUDA's IEEE square root
and division over arguments spanning 2^-1000..2^1000."""
import pytest

from paper_1607_02214_gb300 import ppmlr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1607_02214_gb300 import build
    build.build()


def test_sqrt_and_reciprocal_within_one_ulp():
    err = ppmlr.selftest_fp64_arith(1 << 22)
    print(err)
    assert 0.0 <= err["sqrt_ulp"] <= 1.0
    assert 0.0 <= err["recip_ulp"] <= 1.0


def test_rejects_bad_arguments():
    with pytest.raises(ppmlr.PPMLRError):
        ppmlr.selftest_fp64_arith(0)
