"""The magnitude step (Eq. 4) on the device: the library's F32 magnitude is
sqrtf((float)S) with IEEE rounding, and its U8 magnitude is min(255, round(sqrt S)),
for EVERY S the operator can produce (0 .. 599,270,400 = 4 * 12240^2), and for
every S up to 2^31 - 2 that runtime weights can produce."""
import pytest

import paper_2305_00515_gb300 as pkg

pytestmark = pytest.mark.gpu
S_MAX = 599270400


def test_magnitude_exhaustive():
    from paper_2305_00515_gb300 import build
    build.build()
    st, h = pkg.sobel4_create(0)
    assert st == 0
    try:
        st, bad = pkg.sobel4_check_magnitude(h, 0, S_MAX + 1)
        assert st == 0, pkg.sobel4_status_string(st)
        assert bad == 0, f"{bad} values of S disagree with sqrtf / the exact U8 rule"
        assert pkg.sobel4_check_magnitude(h, 5, 4)[0] == 1
        assert pkg.sobel4_check_magnitude(h, -1, 4)[0] == 1
    finally:
        pkg.sobel4_destroy(h)


def test_magnitude_exhaustive_beyond_eq3():
    """Runtime weights (Eq. 5) can reach S up to 2^31 - 2: the same check there."""
    st, h = pkg.sobel4_create(0)
    assert st == 0
    try:
        st, bad = pkg.sobel4_check_magnitude(h, S_MAX + 1, 2 ** 31 - 1)
        assert st == 0, pkg.sobel4_status_string(st)
        assert bad == 0, f"{bad} values of S disagree with sqrtf / the exact U8 rule"
    finally:
        pkg.sobel4_destroy(h)
