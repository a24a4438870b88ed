"""The integer-pipe FP64 division by 6 equals the device's IEEE division
bit for bit (random bit patterns and every exponent's boundary mantissas)."""
import pytest

from paper_1006_3148_gb300 import jacobi as J

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_exact_division_matches_ieee(seed):
    bad, first = J.jacobi_check_division(1 << 32, seed)
    assert bad == 0, "first failing input 0x%016x" % first
