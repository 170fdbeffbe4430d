"""GPU: carrier recovery through the entry point that allocates nothing.

rx_carrier_recovery_static works in a fixed device array that the library
declares at file scope, for callers that may not allocate device memory while
they process data. Its output must match the carrier-recovered symbols the
regular entry point (rx_process, which works in handle-owned buffers)
produces from the same equalised symbols, on two calls in a row (the second
call reuses the array the first one left behind).
"""

import numpy as np
import pytest

from synth import generate, workload
from tests.gpu_util import rel_rms

pytestmark = pytest.mark.gpu


def _frame_through_rx_process(name, n_sym, seed):
    import torch
    from paper_2011_13695_gb300 import rx
    from paper_2011_13695_gb300.receiver import Receiver
    w = workload(name, n_sym=n_sym)
    fr = generate(w["link"], seed)
    x = np.ascontiguousarray(fr.samples.astype(np.complex64))
    rcv = Receiver(w["rx"], n_sym)
    rcv.process(torch.from_numpy(x.view(np.float32)).cuda(), n_sym)
    y = rcv.buffer(rx.RX_BUF_Y).view(torch.float32).reshape(2, -1, 2)[:, :n_sym].contiguous()
    z = rcv.buffer(rx.RX_BUF_Z).view(torch.float32).reshape(2, -1, 2)[:, :n_sym].contiguous()
    rcv.close()
    return w["rx"], y, z


def _as_complex(t):
    a = t.cpu().numpy()
    return a[..., 0].astype(np.float64) + 1j * a[..., 1]


def test_static_entry_point_matches_rx_process_on_two_calls():
    import torch
    from paper_2011_13695_gb300 import build, rx
    build.build()
    cases = [("dp-qpsk-25gbd", 1 << 14, 1), ("dp-16qam-32gbd", 1 << 15, 2)]
    for name, n, seed in cases:
        rxs, y, z_ref = _frame_through_rx_process(name, n, seed)
        z = torch.full_like(y, float("nan"))
        rx.rx_carrier_recovery_static(y.data_ptr(), n, rxs["bits_per_sym"], rxs["bps_phases"], rxs["bps_window"],
                                      z.data_ptr(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert rel_rms(_as_complex(z), _as_complex(z_ref)) <= 1e-4, name


def test_static_entry_point_rejects_oversized_frames():
    import torch
    from paper_2011_13695_gb300 import build, rx
    build.build()
    t = torch.zeros(16, device="cuda")
    with pytest.raises(rx.RxError) as e:
        rx.rx_carrier_recovery_static(t.data_ptr(), rx.RX_STATIC_MAX_SYMBOLS + 1, 4, 64, 64, t.data_ptr(),
                                      torch.cuda.current_stream().cuda_stream)
    assert e.value.status == rx.RX_EINVAL
