"""The contracted FP64 form's own square root (a float-pair seed, one Newton
step on the exact integer remainder and a final rounding step) equals CUDA's
IEEE square root bit for bit, also on exact squares and their neighbours
a few ulps away; its reciprocal (a float seed, one Newton step on the
exact integer remainder and a final rounding step) equals IEEE division;
its integer-pipe product equals the IEEE product bit for bit on normal
operands with normal results, ties included.  Arguments span
2^-1000..2^1000."""
import pytest

from paper_1607_02214_gb300 import ppmlr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1607_02214_gb300 import build
    build.build()


def test_sqrt_reciprocal_and_product_exact():
    err = ppmlr.selftest_fp64_arith(1 << 24)
    print(err)
    assert err["sqrt_mismatches"] == 0
    assert err["mul_mismatches"] == 0
    assert err["sqrt_ulp"] == 0.0
    assert err["recip_ulp"] == 0.0


def test_rejects_bad_arguments():
    with pytest.raises(ppmlr.PPMLRError):
        ppmlr.selftest_fp64_arith(0)


def test_integer_product_issues_beside_the_fp64_pipe():
    """The integer-pipe product runs at a useful rate alone, and interleaved
    with FP64 FMAs the two together retire more operations per second than
    the FP64 pipe alone (the premise of moving products off it)."""
    co = ppmlr.measure_coissue()
    fp = ppmlr.measure_pipe_rates()
    print(co, fp)
    assert co["int_dmul_per_s"] > 0.5 * fp["dfma_per_s"]
    assert co["dfma_plus_int_dmul_per_s"] > 1.2 * fp["dfma_per_s"]
