"""Host-side knobs of a batched plan (the segment length and task shape the
autotuner picks): defaults, set / get, argument checks. Plans are built from
descriptors with placeholder device addresses; no device memory is touched."""
import ctypes

import pytest

import paper_1303_2285_gb300 as cov


def make_plan(shapes):
    arr = (cov.CovDesc * len(shapes))()
    for k, (N, M, P, Q) in enumerate(shapes):
        arr[k] = cov.CovDesc(0x10000000 + k * 0x100000, 0x40000000 + k * 0x100000, M, N, M, P, Q)
    return cov.BatchedPlan(None, descs=arr)


def test_small_members_default_to_the_warp_form():
    plan = make_plan([(25, 25, 10, 10), (31, 32, 16, 16), (9, 1, 5, 1)])
    assert plan.tuning == {"form": 1, "reseed_interval": 0, "row_ranges": 4}


def test_aperture_sized_members_default_to_the_box_form():
    plan = make_plan([(25, 25, 10, 10), (20, 17, 4, 3), (9, 1, 5, 1)])
    assert plan.tuning == {"form": 2, "reseed_interval": 0, "row_ranges": 4}
    for form in (1, 0, 2):
        plan.set_tuning(form, 0, 4)
        assert plan.tuning["form"] == form


def test_box_form_refused_beyond_its_limits():
    plan = make_plan([(25, 25, 10, 10), (31, 32, 16, 16)])  # PQ = 256 > 100
    with pytest.raises(cov.CovError):
        plan.set_tuning(2)
    plan2 = make_plan([(25, 25, 10, 10), (64, 64, 8, 8)])  # M = 64 > 32
    with pytest.raises(cov.CovError):
        plan2.set_tuning(2)


def test_wide_members_default_to_the_stage_form_and_refuse_the_warp_form():
    plan = make_plan([(25, 25, 10, 10), (64, 64, 8, 8)])  # M = 64 does not fit one warp
    assert plan.tuning == {"form": 3, "reseed_interval": 0, "row_ranges": 4}
    with pytest.raises(cov.CovError):
        plan.set_tuning(1)
    plan.set_tuning(0)  # the CTA form takes them too
    assert plan.tuning["form"] == 0
    plan2 = make_plan([(40, 30, 4, 4)])  # N * M = 1200 > 1024
    assert plan2.tuning["form"] == 3


def test_set_and_get_round_trip():
    plan = make_plan([(25, 25, 10, 10), (20, 17, 4, 3)])
    for form, L, rs in [(0, 3, 2), (0, 0, 1), (1, 0, 4), (0, 16, 4)]:
        plan.set_tuning(form, L, rs)
        assert plan.tuning == {"form": form, "reseed_interval": L, "row_ranges": rs}


@pytest.mark.parametrize("form,L,rs", [(4, 0, 4), (-1, 0, 4), (0, -1, 4), (0, 17, 4), (0, 0, 3),
                                       (0, 0, 0)])
def test_bad_values_are_refused(form, L, rs):
    plan = make_plan([(25, 25, 10, 10)])
    before = plan.tuning
    with pytest.raises(cov.CovError):
        plan.set_tuning(form, L, rs)
    assert plan.tuning == before


def test_stage_form_offered_with_every_other_form():
    plan = make_plan([(25, 25, 10, 10), (64, 64, 8, 8)])
    plan.set_tuning(3)
    assert plan.tuning["form"] == 3
    plan.set_tuning(0)
    assert plan.tuning["form"] == 0


def test_members_only_the_stage_form_takes():
    # P = 20, N < 2P - 1 and M = 600 are beyond the CTA form's limits
    plan = make_plan([(64, 64, 20, 4), (30, 40, 16, 3), (100, 600, 4, 4)])
    assert plan.tuning["form"] == 3
    for form in (0, 1, 2):
        with pytest.raises(cov.CovError):
            plan.set_tuning(form)


def test_null_arguments():
    lib = cov.load()
    t = cov.BatchedTuning()
    assert lib.cov_batched_get_tuning(None, ctypes.byref(t)) != 0
    assert lib.cov_batched_set_tuning(None, ctypes.byref(t)) != 0
    assert lib.cov_batched_autotune(None, None, 0, 1, None) != 0
