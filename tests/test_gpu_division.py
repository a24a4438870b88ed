"""The integer-pipe FP64 division by 6 and FP64 addition equal the device's
IEEE operations bit for bit (random bit patterns, every exponent's boundary
mantissas, and same-sign pairs at every exponent distance)."""
import pytest

from paper_1006_3148_gb300 import jacobi as J

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_exact_division_matches_ieee(seed):
    bad, first = J.jacobi_check_division(1 << 32, seed)
    assert bad == 0, "first failing input 0x%016x" % first


@pytest.mark.parametrize("seed", [1, 2])
def test_exact_integer_addition_matches_ieee(seed):
    bad, first = J.jacobi_check_addition(1 << 30, seed)
    assert bad == 0, "first failing pair 0x%016x + 0x%016x" % first
