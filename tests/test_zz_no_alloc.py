"""GPU: carrier recovery through the entry point that allocates nothing.

rx_carrier_recovery_static works in a fixed device array that the library
declares at file scope, for callers that may not allocate device memory while
they process data (a real-time ingest thread that must not block in the CUDA
allocator; a host framework that fixes the library's memory budget at load
time). The same BPS and unwrap kernels as rx_process run on the same
equalised symbols, so its output must equal the carrier-recovered symbols of
rx_process (which works in handle-owned buffers) bit for bit, on calls in a
row: a 2^14-symbol frame, a 2^15-symbol frame, then a ragged 5003-symbol frame
that runs over the larger frame's leftovers in the shared array. After the
first call (which looks up the array and loads the kernels) the device's free
memory must not change.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _frame_through_rx_process(name, n_sym, seed):
    import torch
    from paper_2011_13695_gb300 import rx
    from paper_2011_13695_gb300.receiver import Receiver
    from synth import generate, workload
    w = workload(name, n_sym=n_sym)
    fr = generate(w["link"], seed)
    x = np.ascontiguousarray(fr.samples.astype(np.complex64))
    rcv = Receiver(w["rx"], n_sym)
    rcv.process(torch.from_numpy(x.view(np.float32)).cuda(), n_sym)
    y = rcv.buffer(rx.RX_BUF_Y).view(torch.float32).reshape(2, -1, 2)[:, :n_sym].contiguous()
    z = rcv.buffer(rx.RX_BUF_Z).view(torch.float32).reshape(2, -1, 2)[:, :n_sym].contiguous()
    rcv.close()
    return w["rx"], y, z


def test_static_entry_point_equals_rx_process_on_three_calls_without_allocating():
    import torch
    from paper_2011_13695_gb300 import build, rx
    build.build()
    cases = [("dp-qpsk-25gbd", 1 << 14, 1), ("dp-16qam-32gbd", 1 << 15, 2), ("dp-16qam-32gbd", 5003, 3)]
    # every reference first: rx_process allocates its handle, the static calls below must not allocate
    frames = [_frame_through_rx_process(name, n, seed) for name, n, seed in cases]
    outs = [torch.full_like(y, float("nan")) for _, y, _ in frames]
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    free = []
    for (name, n, _), (rxs, y, z_ref), z in zip(cases, frames, outs):
        rx.rx_carrier_recovery_static(y.data_ptr(), n, rxs["bits_per_sym"], rxs["bps_phases"], rxs["bps_window"],
                                      z.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        got, want = z.cpu().numpy(), z_ref.cpu().numpy()
        diff = np.flatnonzero(np.any(got != want, axis=-1).ravel())
        assert diff.size == 0, f"{name} n={n}: {diff.size} symbols differ, first {diff[:8]}"
    assert free[1] == free[0] and free[2] == free[0], free


def test_static_entry_point_rejects_oversized_frames():
    import torch
    from paper_2011_13695_gb300 import build, rx
    build.build()
    t = torch.zeros(16, device="cuda")
    with pytest.raises(rx.RxError) as e:
        rx.rx_carrier_recovery_static(t.data_ptr(), rx.RX_STATIC_MAX_SYMBOLS + 1, 4, 64, 64, t.data_ptr(),
                                      torch.cuda.current_stream().cuda_stream)
    assert e.value.status == rx.RX_EINVAL
