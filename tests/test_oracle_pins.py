"""The CPU oracle against the paper's own statements, closed forms and invariants."""
import numpy as np
import pytest

import oracle_checks as oc
from factored_reference import factored_responses


@pytest.mark.parametrize("check", oc.ALL_CHECKS, ids=lambda c: c.__name__)
def test_oracle_pin(oracle_lib, check):
    check(oracle_lib)


@pytest.mark.parametrize("abmn", [(1, 2, 6, 4), (1, 1, 2, 1), (2, 3, 10, 5), (3, 1, 4, 2)])
def test_paper_identities_hold_for_general_weights(abmn):
    """Eq. (10) and Eq. (18) are identities of Eq. (5) for any (a, b, m, n)."""
    a, b, m, n = abmn
    K = oc.eq5_masks(a, b, m, n)
    kp, km = oc.eq10_kd_plus_minus(a, b, m, n)
    assert np.array_equal(K[2] + K[3], kp)
    assert np.array_equal(K[2] - K[3], km)
    assert np.array_equal(oc.eq18_kd_minus(a, b, m, n), km)


def test_factored_path_matches_scipy_for_general_weights():
    """The factored schedule (Eq. 6-19) is exact for other weights too."""
    img = oc.rng_image(9, 21, 26)
    for abmn in ((1, 1, 2, 1), (2, 3, 10, 5)):
        K = oc.eq5_masks(*abmn)
        want = oc.scipy_responses(img, "valid", K)[:, 2:-2, 2:-2]
        for variant in ("eq19", "eq17"):
            got = factored_responses(img, *abmn, kd_minus=variant)
            assert np.array_equal(got, want)


def test_worst_case_range_fits_int32(oracle_lib):
    """|R_k| <= 48*255 and S <= 599,270,400 < 2^31; reached by a checkerboard of 0/255."""
    K = oracle_lib.masks()
    bound = int(np.abs(K).sum(axis=(1, 2)).max() // 2 * 255)
    assert bound == 12240
    assert 4 * bound * bound == 599270400 < 2 ** 31
    I = oc.rng_image(3, 64, 64)
    R = oracle_lib.responses(I, "replicate")
    assert np.abs(R).max() <= 12240


def test_rejects_bad_arguments(oracle_lib):
    with pytest.raises(ValueError):
        oracle_lib.responses(np.zeros((2, 8), np.uint8), "reflect101")
    with pytest.raises(ValueError):
        oracle_lib.sobel4(np.zeros((8, 2), np.uint8), "reflect101")
