"""The C-ABI library builds, loads and exports every entry point of include/fh.h,
and the Python binding's structs match the C layout.  CPU only."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fh.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1407_8333_gb300 import build, fh
    build.build()
    return fh.load()


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fh_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_path_entry_points():
    names = _declared_functions()
    for want in ("fh_create_plan", "fh_correct_doppler", "fh_transform", "fh_select_candidates",
                 "fh_submit", "fh_poll"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1407_8333_gb300 import fh
    names = _declared_functions()
    for n in names:
        assert hasattr(lib, n), n
    # the binding wraps every declared entry point
    assert set(names) <= set(fh.exported_symbols())


def test_struct_layout_matches_c(tmp_path):
    from paper_1407_8333_gb300 import fh
    prog = tmp_path / "layout.c"
    prog.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "fh.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\\n", sizeof(fh_peakmap), sizeof(fh_plan_desc), sizeof(fh_candidate),
         sizeof(fh_job_desc), sizeof(fh_job_stats));
  printf("%zu %zu %zu %zu\\n", offsetof(fh_plan_desc, p0), offsetof(fh_plan_desc, max_peaks),
         offsetof(fh_candidate, f0), offsetof(fh_job_desc, n_dir));
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    got = [int(x) for x in out]
    want = [ctypes.sizeof(fh.fh_peakmap), ctypes.sizeof(fh.fh_plan_desc),
            ctypes.sizeof(fh.fh_candidate), ctypes.sizeof(fh.fh_job_desc),
            ctypes.sizeof(fh.fh_job_stats), fh.fh_plan_desc.p0.offset,
            fh.fh_plan_desc.max_peaks.offset, fh.fh_candidate.f0.offset, fh.fh_job_desc.n_dir.offset]
    assert got == want


def test_invalid_plan_is_rejected_without_gpu(lib):
    """Descriptor validation happens on the host before any CUDA call."""
    from paper_1407_8333_gb300 import fh
    from paper_1407_8333_gb300 import synth
    w = synth.WORKLOADS["nodoppler_T1024_N200_100Hz"]
    pp = dict(w.plan_params())
    pp["k_over"] = 0
    d = fh.make_desc(pp, 10, 1, 100)
    with pytest.raises(fh.FHError) as ei:
        fh.fh_create_plan(d)
    assert ei.value.code == fh.FH_ERR_INVALID_ARG
    assert fh.fh_plan_device_bytes(d) == 0
    pp = dict(w.plan_params())
    d = fh.make_desc(pp, 200, 4, 20000)
    assert fh.fh_plan_device_bytes(d) > 8 * 4 * 20000
    pp["t_fft"] = 1024.0 + 2.0 ** -40   # K * T not exact in binary64
    with pytest.raises(fh.FHError):
        fh.fh_create_plan(fh.make_desc(pp, 10, 1, 100))


def test_selection_workspace_size(lib):
    """fh_peakmap_select_workspace covers a bit per bin and a count per
    4096-bin segment of every FFT, grows with both sizes, and refuses
    negative sizes, without a GPU."""
    f = lib.fh_peakmap_select_workspace
    for n_fft, n_bins in ((1, 1), (3164, 8192), (100, 4097), (65535, 33)):
        ws = f(n_fft, n_bins)
        bits = n_fft * -(-n_bins // 32) * 4
        counts = n_fft * -(-n_bins // 4096) * 4
        assert ws >= bits + counts
        assert f(n_fft + 1, n_bins) >= ws and f(n_fft, n_bins + 4096) >= ws
    assert f(-1, 10) == -1 and f(10, -1) == -1


def test_device_only_outputs_refuse_host_buffers():
    """fh_copy_profile enqueues an asynchronous device-to-device copy: a host
    array is refused before the library is called."""
    import numpy as np
    from paper_1407_8333_gb300 import fh
    with pytest.raises(TypeError):
        fh.fh_copy_profile(None, 0, 1, np.zeros(8, dtype=np.uint64))
    torch = pytest.importorskip("torch")
    with pytest.raises(TypeError):
        fh.fh_copy_profile(None, 0, 1, torch.zeros(8, dtype=torch.int64))


def test_product_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1407_8333_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "fh_oracle" not in txt, f
