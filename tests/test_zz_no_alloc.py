"""The allocation-free check (mc_check_noalloc) against mc_check.

mc_check_noalloc serves callers that cannot allocate device memory (a host
framework that owns the whole device budget, a serving path where an
allocation could block or fail, a plugin limited to a given stream): all its
scratch lives in one static device array of the library.  Its answers must
be bit-identical to mc_check's -- integer work, tolerance zero -- on two
calls in a row, since the array keeps the previous call's contents.  This
file is collected last so that a failure here comes after every other test.
"""
import pytest

from paper_2305_09130_gb300 import workloads as W

pytestmark = pytest.mark.gpu

NO_LIMIT = (1 << 64) - 1


def reference(mc, spec, T, prune, early_exit):
    m = mc.mc_model_create(spec, mc.mc_options_default(prune=prune, early_exit=early_exit))
    r = mc.mc_check(m, T, trace=False)
    mc.mc_model_destroy(m)
    return r


def cases():
    return [W.tiny(W.FREE), W.tiny(W.GREEDY), W.c1(W.FREE), W.c1(W.GREEDY), W.c2(rule=W.GREEDY),
            W.random_small(4242, 5, 3, 2, 6, rule=W.FREE),
            W.random_small(4243, 8, 2, 2, 4, rule=W.GREEDY, key_bits=128)]


def optimum(mc, spec):
    m = mc.mc_model_create(spec)
    t = mc.mc_min_time(m, trace=False)["t_min"]
    mc.mc_model_destroy(m)
    return t


@pytest.mark.parametrize("spec", cases(), ids=lambda s: f"{s.name}_r{s.rule}")
def test_noalloc_matches_mc_check_twice(mc, spec):
    t_min = optimum(mc, spec)
    for T in (t_min - 1, t_min, 3 * t_min, NO_LIMIT):
        for prune, ee in ((True, True), (False, False)):
            exp = reference(mc, spec, T, prune, ee)
            first = mc.mc_check_noalloc(spec, T, prune=prune, early_exit=ee)
            second = mc.mc_check_noalloc(spec, T, prune=prune, early_exit=ee)
            assert first == exp, (T, prune, ee)
            assert second == exp, (T, prune, ee)


def test_noalloc_rejects_models_beyond_its_scratch(mc):
    with pytest.raises(mc.MCError) as e:
        mc.mc_check_noalloc(W.c2_star(), 95)
    assert e.value.code == mc.MC_ERR_NOMEM
    # the array is still usable afterwards
    spec = W.c1(W.FREE)
    assert mc.mc_check_noalloc(spec, 80) == reference(mc, spec, 80, True, True)


def test_noalloc_allocates_no_device_memory(mc):
    """The point of the entry point: a batch of calls leaves the device's
    free memory unchanged (the library's cached pool blocks are given back
    first, and one warm-up call looks the array's address up)."""
    import torch

    spec = W.c1(W.GREEDY)
    t_min = optimum(mc, spec)
    mc.mc_check_noalloc(spec, t_min)
    mc.mc_release_cached()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    answers = [mc.mc_check_noalloc(spec, T, prune=p, early_exit=p)
               for T in (t_min - 1, t_min, NO_LIMIT) for p in (True, False)]
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert [a["holds"] for a in answers] == [True, True, False, False, False, False]
