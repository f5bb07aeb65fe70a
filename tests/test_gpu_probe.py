"""GPU: the FMA peak probe runs every kind, reports the flop it launched and
keeps its chains (the sink holds the value of a chain computed on the host)."""
import numpy as np
import pytest

from gpu_util import dev, tri

pytestmark = pytest.mark.gpu


def test_peak_probe_kinds():
    import torch
    t = tri()
    sink = torch.zeros(2 * 256, dtype=torch.float32, device=dev())
    for kind, lanes in ((0, 1), (1, 2), (2, 1)):
        flop = t.tri_peak_probe(kind, 2, 10, sink)
        torch.cuda.synchronize()
        assert flop == 2 * lanes * 8 * 10 * 2 * 256
        s = sink.cpu().numpy()
        assert np.all(np.isfinite(s))
    # FP64 chains: thread 0 sums a_q = q + 1 after ten steps a = a b + c
    b, c = float(np.float32(0.999999)), float(np.float32(1e-7))
    ref = 0.0
    for q in range(8):
        a = 1.0 + q
        for _ in range(10):
            a = a * b + c
        ref += a
    assert abs(float(s[0]) - ref) <= 1e-5 * ref
    with pytest.raises(t.TriError):
        t.tri_peak_probe(3, 2, 10, sink)
