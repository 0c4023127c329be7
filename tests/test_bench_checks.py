"""The bench's own output checks (host only): they accept the oracle's results
and reject planted mistakes, so a GB/s figure can only come from a correct sort."""
import numpy as np
import pytest

import bench
import oracle
import synth


@pytest.mark.parametrize("dtype", [np.uint16, np.int32, np.float32, np.int64, np.float64])
@pytest.mark.parametrize("desc", [False, True])
def test_checks_accept_the_oracle(dtype, desc):
    keys = synth.random_keys(20_011, dtype, seed=5, mode="dups")
    order = "descending" if desc else "ascending"
    p = oracle.sortperm(keys, order)
    out = oracle.gather(keys, p)
    assert bench.check_sorted(keys, out, desc)
    assert bench.check_perm(keys, p.astype(np.uint32), desc, sorted_out=out)


def test_checks_reject_planted_mistakes():
    keys = synth.normal_f32_special(10_007, seed=9, frac=0.02)
    p = oracle.sortperm(keys)
    out = oracle.gather(keys, p)
    # two neighbours swapped: out of order
    bad = out.copy()
    bad[[100, 101]] = bad[[101, 100]]
    if bench._order_key(bad[100:101])[0] != bench._order_key(bad[101:102])[0]:
        assert not bench.check_sorted(keys, bad)
    # one key replaced by its neighbour: sorted, but not the input's multiset
    dup = out.copy()
    dup[200] = dup[199]
    assert not bench.check_sorted(keys, dup)
    # -0.0 after +0.0 is out of Julia's order
    z = np.array([0.0, -0.0], dtype=np.float32)
    assert not bench.check_sorted(z, z)
    assert bench.check_sorted(z, z[::-1].copy())
    # two NaNs (equivalent keys) swapped in the permutation: sorted, same
    # multiset, but not stable
    ties = np.where(np.isnan(out))[0]
    assert ties.size >= 2
    q = p.copy()
    q[[ties[0], ties[1]]] = q[[ties[1], ties[0]]]
    assert not bench.check_perm(keys, q.astype(np.uint32))
    # not a permutation
    r = p.copy()
    r[0] = r[1]
    assert not bench.check_perm(keys, r.astype(np.uint32))
    # a permutation whose gather disagrees with the returned keys
    assert not bench.check_perm(keys, p.astype(np.uint32), sorted_out=dup)


def test_scan_checks_accept_the_oracle_and_reject_planted_mistakes():
    """The accumulate workload's output checks: the oracle's inclusive + passes
    both; a dropped key, a repeated key and two swapped outputs fail."""
    x = synth.uniform_i64(50_021, seed=117)
    good = oracle.accumulate(x, "add")
    assert bench.check_scan_i64(x, good)
    dropped = good.copy()
    with np.errstate(over="ignore"):
        dropped[300:] -= x[300]
    assert not bench.check_scan_i64(x, dropped)
    xf = synth.dist_f64(50_021, "normal", seed=118)
    gf = oracle.accumulate(xf, "add")
    assert bench.check_scan_f64(xf, gf)
    rep = gf.copy()
    rep[7000:] += xf[6999]  # key 6999 counted twice
    assert not bench.check_scan_f64(xf, rep)
    sw = gf.copy()
    sw[[40, 41]] = sw[[41, 40]]
    assert not bench.check_scan_f64(xf, sw)


def test_cpu_list_parsing_and_unbound_fallback():
    """The GPU-local CPU list of sysfs ('0-3,8,10-11'), and the binding that
    leaves the process alone when the device has no sysfs entry."""
    assert bench._cpulist("0-3,8,10-11\n") == {0, 1, 2, 3, 8, 10, 11}
    assert bench._cpulist("") == set()

    class Props:
        pci_domain_id, pci_bus_id, pci_device_id = 0x7FFF, 0xFE, 0x1F

    class FakeTorch:
        class cuda:
            @staticmethod
            def get_device_properties(dev):
                return Props()

    import os
    before = os.sched_getaffinity(0)
    assert "unbound" in bench.bind_to_gpu_node(FakeTorch, 0)
    assert os.sched_getaffinity(0) == before
