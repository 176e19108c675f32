"""perc_nstar_noalloc, the entry point for callers that cannot allocate device memory.

Such callers (for example code that runs inside a framework which owns every device allocation,
or that has to stay within a memory budget fixed in advance) cannot hand the library a workspace.
perc_nstar_noalloc uses a fixed array that the library itself keeps in device memory instead.  These
tests call it through the C ABI and check that two calls in a row return exactly what perc_nstar
returns on the same samples and what the oracle's Newman--Ziff sweep gives; this file is named so
that pytest collects it last.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


def _samples(L, masks, seeds):
    from paper_2607_18991_b300 import perc
    perm, rk = perc.rank(L, seeds)
    masks_all = [m for s in range(len(seeds)) for m in masks]
    rows = [s for s in range(len(seeds)) for _ in masks]
    return perc.samples_for(L, masks_all, rows, perm, rk), (perm, rk)


@pytest.mark.parametrize("L,masks,seeds", [(8, list(range(1, 128, 5)), [1, 2, 3]),
                                           (16, [1, 7, 42, 127], [4, 5])])
def test_noalloc_matches_workspace_entry_point_twice(L, masks, seeds):
    import torch

    from paper_2607_18991_b300 import perc
    smp, keep = _samples(L, masks, seeds)
    perc.set_launch_option(perc.OPT_METHOD, perc.METHOD_BISECTION)  # the method the no-alloc entry uses
    try:
        want_ns, want_ps = perc.nstar(smp, L)
    finally:
        perc.set_launch_option(perc.OPT_METHOD, perc.METHOD_AUTO)
    want_ns, want_ps = perc.u32(want_ns), perc.u32(want_ps)
    N = L ** 5
    exact = torch.from_numpy(np.stack([want_ns, want_ns], axis=1).astype(np.uint32).view(np.int32)).cuda()
    for _ in range(2):  # the static scratch keeps the previous call's contents; results must not depend on it
        ns, ps = perc.nstar_noalloc(smp, L)
        assert np.array_equal(perc.u32(ns), want_ns)
        assert np.array_equal(perc.u32(ps), want_ps)
        ns_b, _ = perc.nstar_noalloc(smp, L, bracket=exact)
        assert np.array_equal(perc.u32(ns_b), want_ns)
    assert np.all(want_ns <= N)
    orc = [oracle.nz(L, m, *oracle.rank(L, s))[0] for s in seeds for m in masks]
    assert np.array_equal(want_ns, np.array(orc, dtype=np.uint32))
    torch.cuda.synchronize()


def test_noalloc_largest_lattice_that_fits():
    """L = 23 is the largest side whose one CTA slot (about 57 MiB) fits in the 64 MiB scratch."""
    from paper_2607_18991_b300 import perc
    smp, keep = _samples(23, [127], [1])
    for _ in range(2):
        ns, _ = perc.nstar_noalloc(smp, 23)
        assert perc.u32(ns)[0] == oracle.nz(23, 127, *oracle.rank(23, 1))[0]


def test_noalloc_rejects_lattices_beyond_its_scratch():
    from paper_2607_18991_b300 import perc
    smp, keep = _samples(4, [1], [1])
    for max_L in (24, 40):  # one CTA slot: about 69 MiB at L = 24, far more at L = 40
        with pytest.raises(perc.PercError) as err:
            perc.nstar_noalloc(smp, max_L)
        assert err.value.rc == -2
