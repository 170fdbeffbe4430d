"""GPU parity of the learned post-equaliser (BF16 kernels through the rx_pe C ABI)
against the FP64 oracle network.

Precision reading: the kernels store weights and activations in BF16 and
accumulate in FP32. The oracle is given the same BF16-rounded parameters and
BF16-rounded input channels, so what remains is the rounding of the three
hidden activations to BF16 (relative 2^-9 each, uniform, RMS 2^-9/sqrt(3))
propagated through the following layers, plus FP32 accumulation over
64 x 9 = 576 terms. Three such roundings give about 0.2 % relative RMS on
f(z); the tests allow 1 %. Gradients carry the same activation roundings in
their factors: 2 % per tensor and a cosine above 0.999.
"""

from __future__ import annotations

import numpy as np
import pytest

from oracle import cnn

pytestmark = pytest.mark.gpu

C, K = 64, 9


def bf16(a: np.ndarray) -> np.ndarray:
    """Round to the nearest BF16 (ties to even), returned as float64."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def random_params(seed: int) -> list:
    rng = np.random.default_rng(seed)
    params = cnn.init_params(C, K, seed=seed, out_scale=1.0)
    for layer in params:
        layer[1] = rng.normal(0.0, 0.1, size=layer[1].shape)
    return params


def channels(zc: np.ndarray) -> np.ndarray:
    """complex [2, T] -> real [4, T] (I_x, Q_x, I_y, Q_y)."""
    return np.stack([zc[0].real, zc[0].imag, zc[1].real, zc[1].imag])


def qam_like(T: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    lv = np.array([-3.0, -1.0, 1.0, 3.0]) / np.sqrt(10.0)
    s = lv[rng.integers(0, 4, size=(2, T))] + 1j * lv[rng.integers(0, 4, size=(2, T))]
    return s + 0.1 * (rng.standard_normal((2, T)) + 1j * rng.standard_normal((2, T)))


def oracle_f(params_bf16: list, zc: np.ndarray) -> np.ndarray:
    """f(z) of the oracle on BF16-rounded input channels (the residual is added with the FP32 input)."""
    x = bf16(channels(zc))
    out, _ = cnn.forward(params_bf16, x)
    return out - x


def rel(a, b) -> float:
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def to_dev(zc: np.ndarray):
    import torch
    return torch.from_numpy(np.ascontiguousarray(zc.astype(np.complex64))).cuda()


@pytest.fixture(scope="module")
def pe_params():
    params = random_params(11)
    vec = cnn.flatten(params).astype(np.float32)
    return vec, cnn.unflatten(bf16(vec), C, K)


# 128 (input layer) and 248 (hidden and output layers) positions per tile: lengths at and around
# the tile boundaries, and one that ends a tile one position into it
@pytest.mark.parametrize("T", [1, 7, 127, 128, 129, 247, 248, 249, 300, 496, 497, 3001, 4096])
def test_forward_matches_oracle(pe_params, T):
    from paper_2011_13695_gb300.learned import PostEqualiser
    vec, pb = pe_params
    zc = qam_like(T, seed=T)
    pe = PostEqualiser(4096, vec)
    out = pe.forward(to_dev(zc)).cpu().numpy().astype(np.complex128)
    assert pe.error_word() == 0
    pe.close()
    zf = zc.astype(np.complex64).astype(np.complex128)
    f_gpu = channels(out - zf)
    f_ref = oracle_f(pb, zc)
    assert rel(f_gpu, f_ref) < 1e-2, rel(f_gpu, f_ref)


def test_forward_full_length_sampled(pe_params):
    """At the largest sequence (2^20 symbols), windows checked against the oracle on a slice with
    16 symbols of context on each side (the receptive field: 4 layers x 4); the two sequence ends
    check the zero padding."""
    from paper_2011_13695_gb300.learned import PostEqualiser
    vec, pb = pe_params
    T = 1 << 20
    zc = qam_like(T, seed=5)
    pe = PostEqualiser(T, vec)
    out = pe.forward(to_dev(zc)).cpu().numpy().astype(np.complex128)
    assert pe.error_word() == 0
    pe.close()
    zf = zc.astype(np.complex64).astype(np.complex128)
    R, w = 16, 512
    for a in (0, 12345, T // 2 + 7, T - w):
        lo, hi = max(0, a - R), min(T, a + w + R)
        f_ref = oracle_f(pb, zc[:, lo:hi])[:, a - lo:a - lo + w]
        f_gpu = channels(out[:, a:a + w] - zf[:, a:a + w])
        assert rel(f_gpu, f_ref) < 1e-2, (a, rel(f_gpu, f_ref))


@pytest.mark.parametrize("T", [9, 2999])
def test_gradients_match_oracle(pe_params, T):
    from paper_2011_13695_gb300.learned import PostEqualiser
    vec, pb = pe_params
    zc = qam_like(T, seed=100 + T)
    tc = qam_like(T, seed=200 + T)
    pe = PostEqualiser(4096, vec)
    g_dev, loss_dev = pe.gradients(to_dev(zc), to_dev(tc))
    g = g_dev.cpu().numpy().astype(np.float64)
    loss = float(loss_dev.cpu().item())
    pe.close()
    x = bf16(channels(zc))
    out, acts = cnn.forward(pb, x)
    # the kernel's residual adds the FP32 input, not its BF16 copy
    out = out - x + channels(zc.astype(np.complex64).astype(np.complex128))
    tgt = channels(tc.astype(np.complex64).astype(np.complex128))
    assert abs(loss - cnn.mse(out, tgt)) <= 1e-2 * cnn.mse(out, tgt)
    ref = cnn.backward(pb, acts, out, tgt)
    got = cnn.unflatten(g, C, K)
    for li in range(cnn.LAYERS):
        for j in range(2):
            a, b = got[li][j].ravel(), ref[li][j].ravel()
            cos = float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b)))
            assert rel(a, b) < 2e-2 and cos > 0.999, (li, j, rel(a, b), cos)


def test_adam_step_matches_oracle(pe_params):
    """One training step: the update applied to the FP32 master weights equals the oracle's Adam
    step on the same gradients (taken from the kernels, so only the optimiser is compared)."""
    from paper_2011_13695_gb300.learned import PostEqualiser
    vec, _ = pe_params
    T = 1500
    zc, tc = qam_like(T, seed=1), qam_like(T, seed=2)
    pe = PostEqualiser(4096, vec)
    z, t = to_dev(zc), to_dev(tc)
    g = pe.gradients(z, t)[0].cpu().numpy().astype(np.float64)
    lr = 1e-3
    pe.train_step(z, t, lr)
    p1 = pe.params().astype(np.float64)
    pe.close()
    params = cnn.unflatten(vec.astype(np.float64), C, K)
    opt = cnn.Adam(params, lr=lr)
    ref = cnn.flatten(opt.step(params, cnn.unflatten(g, C, K)))
    # first Adam step moves each weight by lr * g / (|g| + eps): compare where |g| is well above the
    # run-to-run change of the atomically accumulated gradient
    big = np.abs(g) > 1e-4 * np.abs(g).max()
    assert np.max(np.abs(p1 - ref)[big]) <= 1e-3 * lr + 1e-6 * np.abs(ref[big]).max()
    assert np.max(np.abs(p1 - vec)) <= lr * 1.001 + 1e-7


def test_training_reduces_loss():
    """A fixed linear inter-symbol interference (each symbol picks up 0.25 j times its predecessor) is
    learnable through the residual ReLU network: 400 Adam steps on 4096-symbol slices bring the MSE
    to a small fraction of the identity's. The rate decays from 2e-3 to 2e-4 so that the weights
    the inference forward is judged on are not taken at a spike of the last steps (at a constant
    2e-3 the final weights scored between 5 % and 15 % of the identity's MSE from run to run, the
    weight gradients' atomic sums making runs differ)."""
    import torch
    from paper_2011_13695_gb300.learned import PostEqualiser
    rng = np.random.default_rng(7)
    T = 1 << 16
    lv = np.array([-3.0, -1.0, 1.0, 3.0]) / np.sqrt(10.0)
    s = lv[rng.integers(0, 4, size=(2, T))] + 1j * lv[rng.integers(0, 4, size=(2, T))]
    zc = s + 0.25j * np.roll(s, 1, axis=1) + 0.02 * (rng.standard_normal((2, T)) + 1j * rng.standard_normal((2, T)))
    params = cnn.init_params(C, K, seed=3)
    pe = PostEqualiser(4096, cnn.flatten(params).astype(np.float32))
    z, t = to_dev(zc), to_dev(s)
    losses = pe.train(z, t, 0, T, steps=400, window=4096, lr=2e-3, seed=1, lr_final=2e-4)
    out = pe.forward(z[:, :4096].contiguous())
    pe.close()
    l0 = float(np.mean(np.abs(zc[:, :4096] - s[:, :4096]) ** 2)) / 2
    l_end = float(torch.mean(torch.abs(out - t[:, :4096]) ** 2).item()) / 2
    first = float(losses[:10].mean().item())
    last = float(losses[-10:].mean().item())
    assert torch.isfinite(losses).all()
    assert last < 0.1 * first and l_end < 0.1 * l0, (first, last, l0, l_end)


def test_train_steps_equal_single_steps():
    """rx_pe_train_steps (the whole schedule in one call, windows read in place from two sequences of
    different lengths) leaves the same parameters, bit for bit, as one rx_pe_train_step per step on
    contiguous copies of the same windows with the same rates (the update's kernels are deterministic),
    and the same losses to rounding."""
    import torch
    from paper_2011_13695_gb300 import rx
    from paper_2011_13695_gb300.learned import PostEqualiser
    n = [5000, 3100]
    zs = [to_dev(qam_like(v, seed=31 + i)) for i, v in enumerate(n)]
    ts = [to_dev(qam_like(v, seed=41 + i)) for i, v in enumerate(n)]
    params = cnn.flatten(cnn.init_params(C, K, seed=5)).astype(np.float32)
    rng = np.random.default_rng(9)
    W, steps = 1024, 12
    which = rng.integers(0, 2, size=steps)
    offs = [int(rng.integers(0, n[k] - W + 1)) for k in which]
    lrs = [1e-3 * 0.9 ** i for i in range(steps)]
    a = PostEqualiser(4096, params)
    la = torch.zeros(steps, dtype=torch.float32, device="cuda")
    rx.rx_pe_train_steps(a.h, [v.data_ptr() for v in zs], [v.data_ptr() for v in ts], n, W, which, offs, lrs,
                         la.data_ptr(), torch.cuda.current_stream().cuda_stream)
    b = PostEqualiser(4096, params)
    lb = torch.zeros(steps, dtype=torch.float32, device="cuda")
    for i, k in enumerate(which):
        zw = zs[k][:, offs[i]:offs[i] + W].contiguous()
        tw = ts[k][:, offs[i]:offs[i] + W].contiguous()
        b.train_step(zw, tw, lrs[i], lb.data_ptr() + 4 * i)
    pa, pb = a.params(), b.params()
    assert a.error_word() == 0 and b.error_word() == 0
    with pytest.raises(rx.RxError):                  # a window past the end of its sequence
        rx.rx_pe_train_steps(a.h, [zs[0].data_ptr()], [ts[0].data_ptr()], [n[0]], W, [0], [n[0] - W + 1], [1e-3],
                             None, None)
    a.close()
    b.close()
    assert np.array_equal(pa, pb), float(np.max(np.abs(pa - pb)))
    # the reported loss is summed with float atomics across warps (it feeds no update): equal to rounding
    assert torch.allclose(la, lb, rtol=1e-5, atol=0.0), (la, lb)


def test_inference_forward_equals_training_forward():
    """The inference forward (tensor cores, channel-chunk planes) and the training forward (channel-major
    activations) compute the same network: after some training, the loss of the inference output equals
    the loss the gradient call computes from its own forward on the same window (both accumulate in FP32
    over BF16 operands, in different orders)."""
    import torch
    from paper_2011_13695_gb300.learned import PostEqualiser
    T = 3001
    zc, tc = qam_like(T, seed=21), qam_like(T, seed=22)
    params = cnn.init_params(C, K, seed=4)
    pe = PostEqualiser(4096, cnn.flatten(params).astype(np.float32))
    z, t = to_dev(zc), to_dev(tc)
    pe.train(z, t, 0, T, steps=30, window=2048, lr=1e-3, seed=2)
    out = pe.forward(z)
    l_inf = float(torch.mean(torch.abs(out - t) ** 2).item()) / 2
    _, loss = pe.gradients(z, t)
    l_tr = float(loss.item())
    assert pe.error_word() == 0
    pe.close()
    assert abs(l_inf - l_tr) <= 1e-4 * l_tr, (l_inf, l_tr)


def test_invalid_arguments():
    import torch
    from paper_2011_13695_gb300 import rx
    from paper_2011_13695_gb300.learned import PostEqualiser
    assert rx.rx_pe_param_count(32, 9) == -1
    assert rx.rx_pe_param_count(64, 9) == cnn.flatten(cnn.init_params(C, K)).size
    pe = PostEqualiser(64)
    z = torch.zeros((2, 65), dtype=torch.complex64, device="cuda")
    with pytest.raises(rx.RxError):
        pe.forward(z)
    pe.close()
