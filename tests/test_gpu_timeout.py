"""The bounded waits of the tensor-core kernels give up cleanly (needs a GPU).

Every mbarrier wait in the tcgen05 kernels is limited by %globaltimer. The
diagnostic entry point tachiom_debug_wait_timeout runs one CTA of the step (a)
tensor-core pass whose TMA producer issues no copy, with the limit shortened
to a few milliseconds: its first wait must run out, raise
TACHIOM_FLAG_TIMEOUT, free TMEM and return, long before the usual 2 s limit,
and the device must stay usable (a following search returns the FP32 path's
results).
"""
import time

import numpy as np
import pytest

from test_gpu_parity import _cuda, _search, _tc, get_case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_the_device_stays_usable():
    _cuda()
    _tc()
    c = get_case("small")
    c.G.stream_status()  # clear
    t0 = time.perf_counter()
    c.G.debug_wait_timeout(3000)  # 3 ms
    fl = c.G.stream_status()
    dt = time.perf_counter() - t0
    assert fl & 16, fl  # TACHIOM_FLAG_TIMEOUT
    assert dt < 1.0, dt  # gave up at the short limit, not the default 2 s
    a = _search(c, prec=1)
    b = _search(c, prec=0)
    assert np.array_equal(a[0], b[0])
    assert np.array_equal(a[1].view(np.int32), b[1].view(np.int32))
    assert c.G.stream_status() == 0
