"""qs_set_amps from page-locked host memory (read by the SM copy kernel
through the mapped pointer) and from pageable memory (the copy engine) give
the same device state: whole ranges, partial ranges at aligned and unaligned
offsets (unaligned ones fall back to the copy engine), both precisions."""

import numpy as np
import pytest
import torch

from paper_2311_01512_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qs():
    from paper_2311_01512_gb300 import qs as mod
    return mod


@pytest.mark.parametrize("prec", [0, 1])
def test_set_amps_page_locked_matches_pageable(qs, prec):
    nq = 20                                   # 8 or 16 MiB: above the 1 MiB threshold
    dt = np.complex64 if prec == 0 else np.complex128
    host = wl.random_statevector(nq, np.random.default_rng(77 + prec)).astype(dt)
    pinned = torch.from_numpy(host).pin_memory()
    assert pinned.is_pinned()
    n = 1 << nq
    st = qs.State(nq, prec=prec)
    qs.qs_set_amps_ptr(st.handle, pinned.data_ptr(), 0, n)
    assert np.array_equal(st.get_amps(), host)
    # (aligned start and size; odd start and size; the upper half; below the threshold)
    for first, count in [(1 << 18, 1 << 17), (3, (1 << 19) + 5), (n // 2, n // 2), (7, 1000)]:
        st.set_amps(np.zeros(n, dtype=dt))
        qs.qs_set_amps_ptr(st.handle, pinned.data_ptr() + first * host.itemsize, first, count)
        want = np.zeros(n, dtype=dt)
        want[first:first + count] = host[first:first + count]
        assert np.array_equal(st.get_amps(), want), (first, count)
    # pageable source, same result
    st.set_amps(np.zeros(n, dtype=dt))
    st.set_amps(host)
    assert np.array_equal(st.get_amps(), host)
    st.close()
