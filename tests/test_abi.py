"""CPU checks of the C ABI: the library builds, loads and exports every declared symbol,
and the ctypes mirrors of the structs have the C layout (no GPU needed)."""

import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rx.h")


@pytest.fixture(scope="module")
def librx():
    from paper_2011_13695_gb300 import build, rx
    build.build()
    return rx.lib()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rx_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("rx_create", "rx_process", "rx_stats", "rx_destroy", "rx_process_host", "rx_get_buffer",
                 "rx_state_get", "rx_state_set", "rx_reset", "rx_strerror"):
        assert must in names


def test_library_exports_every_declared_symbol(librx):
    from paper_2011_13695_gb300 import rx
    for name in declared_functions():
        assert hasattr(librx, name), name
    assert set(rx.EXPORTS) == set(declared_functions())


def test_status_strings_without_a_gpu(librx):
    from paper_2011_13695_gb300 import rx
    assert rx.rx_strerror(rx.RX_OK) == "ok"
    assert "invalid" in rx.rx_strerror(rx.RX_EINVAL)
    assert rx.rx_stage_count() == len([rx.rx_stage_name(i) for i in range(rx.rx_stage_count())])
    assert rx.rx_stage_name(1) == "cdc"


def test_invalid_configs_are_rejected_before_any_device_call(librx):
    from paper_2011_13695_gb300 import rx
    base = dict(bits_per_sym=4, sps=2, symbol_rate_hz=32e9, wavelength_m=1550e-9, dispersion_s_per_m2=17e-6,
                length_m=80e3, rrc_rolloff=0.1, fft_size=4096, n_taps=21, lms_block=128, cma_blocks=64,
                dd_acq_blocks=128, seg_blocks=16, warmup_blocks=4, bps_phases=64, bps_window=64, edge_skip=512,
                sync_len=4096, max_delay=16, mu_cma=1e-3, mu_dd=1e-3, fo_grid_hz=100e3, input_format=0,
                input_scale=1.0, streaming=0, max_symbols=1 << 16)
    bad = [dict(sps=4), dict(bits_per_sym=3), dict(fft_size=3000), dict(fft_size=16384), dict(n_taps=20),
           dict(n_taps=65), dict(lms_block=8), dict(bps_phases=65), dict(bps_window=48), dict(max_delay=65),
           dict(warmup_blocks=17), dict(max_symbols=0), dict(input_format=3), dict(symbol_rate_hz=0.0),
           dict(cma_blocks=200), dict(streaming=1, max_symbols=1000), dict(fo_grid_hz=0.0), dict(mu_dd=-1.0)]
    for b in bad:
        with pytest.raises(rx.RxError) as e:
            rx.rx_create(rx.make_config(**dict(base, **b)))
        assert e.value.status == rx.RX_EINVAL, b


def test_widely_linear_stage_rejects_bad_arguments_before_any_device_call(librx):
    from paper_2011_13695_gb300 import rx
    fake = 1 << 20          # never dereferenced: every case fails validation first
    base = dict(d_x=fake, x_len=4096, n_taps=21, d_taps_in=fake, n_sym=2048, block_len=64, seg_blocks=16,
                warmup_blocks=4, bits_per_sym=4, mu=1e-3, mu_conj=1e-3, d_y=fake, d_taps_out=None, threads=0,
                stream=None)
    taps_bytes = 2 * 4 * 21 * 8
    bad = [dict(d_x=0), dict(d_y=0), dict(d_taps_in=0), dict(n_sym=0), dict(x_len=0), dict(n_taps=20),
           dict(n_taps=65), dict(n_taps=1), dict(block_len=8), dict(block_len=512), dict(seg_blocks=0),
           dict(warmup_blocks=-1), dict(bits_per_sym=3), dict(d_taps_out=fake + taps_bytes - 8),
           dict(d_taps_out=fake - taps_bytes + 8), dict(n_sym=1 << 40, seg_blocks=1, block_len=16),
           dict(threads=64), dict(threads=300), dict(threads=128, n_taps=23), dict(threads=256, n_taps=65),
           dict(threads=128, seg_blocks=300)]
    for b in bad:
        with pytest.raises(rx.RxError) as e:
            rx.rx_dd_lms_wl(**dict(base, **b))
        assert e.value.status == rx.RX_EINVAL, b


def test_kk_front_end_rejects_bad_arguments_before_any_device_call(librx):
    from paper_2011_13695_gb300 import rx
    base = dict(fft_size=1024, tone_over_fs=0.13675, rrc_rolloff=0.01, code_scale=1e-3, dc_offset=0.5,
                min_intensity=1e-6)
    bad = [dict(fft_size=512), dict(fft_size=1000), dict(fft_size=16384), dict(tone_over_fs=0.0),
           dict(tone_over_fs=0.5), dict(rrc_rolloff=0.0), dict(rrc_rolloff=1.5), dict(code_scale=0.0),
           dict(code_scale=float("nan")), dict(dc_offset=float("inf")), dict(min_intensity=0.0)]
    for b in bad:
        with pytest.raises(rx.RxError) as e:
            rx.rx_kk_create(**dict(base, **b))
        assert e.value.status == rx.RX_EINVAL, b
    fake = 1 << 20
    for args in [(0, fake, 1024, 0, fake, fake), (fake, 0, 1024, 0, fake, fake), (fake, fake, 1023, 0, fake, fake),
                 (fake, fake + 2, 1024, 0, fake, fake),
                 (fake, fake, 0, 0, fake, fake), (fake, fake, 1024, 0, 0, fake), (fake, fake, 1024, 0, fake, 0)]:
        with pytest.raises(rx.RxError) as e:
            rx.rx_kk_process(*args, None)
        assert e.value.status == rx.RX_EINVAL, args


def test_pam_chain_rejects_bad_arguments_before_any_device_call(librx):
    from paper_2011_13695_gb300 import rx
    base = dict(fft_size=1024, levels=4, rrc_rolloff=0.5, code_scale=1e-3, dc_offset=0.5, max_samples=1 << 20)
    bad = [dict(fft_size=512), dict(fft_size=8192), dict(fft_size=1000), dict(levels=3), dict(levels=16),
           dict(rrc_rolloff=0.0), dict(rrc_rolloff=1.5), dict(code_scale=0.0), dict(dc_offset=float("nan")),
           dict(max_samples=1), dict(max_samples=(1 << 30) + 2)]
    for b in bad:
        with pytest.raises(rx.RxError) as e:
            rx.rx_pam_create(**dict(base, **b))
        assert e.value.status == rx.RX_EINVAL, b
    fake = 1 << 20
    for args in [(0, fake, 1024, fake, fake, fake), (fake, 0, 1024, fake, fake, fake),
                 (fake, fake, 1024, 0, fake, fake), (fake, fake, 1024, fake, 0, fake),
                 (fake, fake, 1024, fake, fake, 0)]:
        with pytest.raises(rx.RxError) as e:
            rx.rx_pam_process(*args, None)
        assert e.value.status == rx.RX_EINVAL, args


def test_ingest_rejects_missing_arguments_before_any_device_call(librx):
    import numpy as np
    from paper_2011_13695_gb300 import rx
    src = np.zeros(4096, dtype=np.uint16)
    st = rx.rx_ingest_stats()
    lib = rx.lib()
    assert lib.rx_ingest_run(None, src.ctypes.data, 4096, 4096, 4e9, 2, 1, None, ctypes.byref(st)) == rx.RX_EINVAL
    assert lib.rx_ingest_run(1 << 20, None, 4096, 4096, 4e9, 2, 1, None, ctypes.byref(st)) == rx.RX_EINVAL
    assert lib.rx_ingest_run(1 << 20, src.ctypes.data, 4096, 4096, 4e9, 2, 1, None, None) == rx.RX_EINVAL


def test_struct_layout_matches_the_c_compiler(librx):
    from paper_2011_13695_gb300 import rx
    fields = [n for n, _ in rx.rx_config._fields_]
    sfields = [n for n, _ in rx.rx_stats_t._fields_]
    ifields = [n for n, _ in rx.rx_ingest_stats._fields_]
    prog = ["#include <stdio.h>", "#include <stddef.h>", f'#include "{HEADER}"', "int main(void){",
            'printf("%zu %zu %zu\\n", sizeof(rx_config), sizeof(rx_stats_t), sizeof(rx_ingest_stats));']
    prog += [f'printf("%zu\\n", offsetof(rx_config, {f}));' for f in fields]
    prog += [f'printf("%zu\\n", offsetof(rx_stats_t, {f}));' for f in sfields]
    prog += [f'printf("%zu\\n", offsetof(rx_ingest_stats, {f}));' for f in ifields]
    prog += ["return 0;}"]
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write("\n".join(prog))
        exe = os.path.join(d, "t")
        subprocess.run(["gcc", "-std=c99", "-o", exe, c], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    vals = list(map(int, out))
    assert vals[0] == ctypes.sizeof(rx.rx_config) and vals[1] == ctypes.sizeof(rx.rx_stats_t)
    assert vals[2] == ctypes.sizeof(rx.rx_ingest_stats)
    offs = vals[3:]
    n1, n2 = len(fields), len(fields) + len(sfields)
    assert offs[:n1] == [getattr(rx.rx_config, f).offset for f in fields]
    assert offs[n1:n2] == [getattr(rx.rx_stats_t, f).offset for f in sfields]
    assert offs[n2:] == [getattr(rx.rx_ingest_stats, f).offset for f in ifields]
