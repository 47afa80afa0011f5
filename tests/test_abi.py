"""The C-ABI library loads on any machine and exports what include/spg.h
declares (no compute: these run without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "spg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(spg_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    import paper_2502_02317_gb300 as spg
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(spg.lib, n), n


def test_params_defaults_and_struct_layout():
    import paper_2502_02317_gb300 as spg
    from paper_2502_02317_gb300 import _binding as b
    p = spg.params()
    assert (p.beta, p.chi, p.beam, p.num_sweeps, p.precision, p.merge, p.svd_iters) == (1.0, 16, 256, 0, 0, 1, -1)
    assert ctypes.sizeof(b.spg_params) == 80
    assert ctypes.sizeof(b.spg_info) == 88
    assert (p.fp64_rows, p.check_fp64, p.group_max) == (-1, 0, 0)
    assert spg.lib.spg_version() == 100
    assert spg.lib.spg_params_default(None) == b.SPG_EINVAL


def test_no_device_is_a_loud_error():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    import paper_2502_02317_gb300 as spg
    with pytest.raises(spg.SpgError):
        spg.Context(0)


def _run(code, env):
    import subprocess
    import sys
    out = subprocess.run([sys.executable, "-c", code], env=env, cwd=ROOT, capture_output=True, text=True,
                         timeout=300)
    assert out.returncode == 0, out.stderr
    return out.stdout.strip()


def test_batch_streams_get_their_own_hardware_queues():
    """spg_solve_batch overlaps up to 32 worker streams, which needs as many
    hardware work queues: the package and the library both ask for 32 unless
    the user chose a value."""
    env = {k: v for k, v in os.environ.items() if k != "CUDA_DEVICE_MAX_CONNECTIONS"}
    assert _run("import os, paper_2502_02317_gb300; print(os.environ['CUDA_DEVICE_MAX_CONNECTIONS'])", env) == "32"
    # the library alone, loaded without the package (C environment, read
    # back through libc)
    import paper_2502_02317_gb300 as spg  # builds the library if needed
    lib = spg.lib._name
    code = ("import ctypes; ctypes.CDLL(%r); "
            "libc = ctypes.CDLL(None); libc.getenv.restype = ctypes.c_char_p; "
            "print(libc.getenv(b'CUDA_DEVICE_MAX_CONNECTIONS').decode())") % lib
    assert _run(code, env) == "32"
    env["CUDA_DEVICE_MAX_CONNECTIONS"] = "8"
    assert _run("import os, paper_2502_02317_gb300; print(os.environ['CUDA_DEVICE_MAX_CONNECTIONS'])", env) == "8"
    assert _run(code, env) == "8"


@pytest.mark.parametrize("rows,cols", [(3, 3), (3, 5), (1, 4), (16, 16), (6, 12)])
def test_lattice_site_map_matches_the_oracle(rows, cols):
    """spg_lattice_site_map (host only) against the oracle's transformation
    of grid positions, for all 8 transformations."""
    import paper_2502_02317_gb300 as spg
    from oracle import lattice
    for k in range(8):
        m, R, C = spg.spg_lattice_site_map(rows, cols, k)
        _, _, R2, C2 = lattice.position(0, 0, rows, cols, k)
        assert (R, C) == (R2, C2)
        assert m.tolist() == lattice.site_map(rows, cols, k).tolist()


def test_lattice_site_map_rejects_bad_arguments():
    import paper_2502_02317_gb300 as spg
    for args in [(0, 3, 0), (3, 0, 0), (3, 3, 8), (3, 3, -1)]:
        with pytest.raises(spg.SpgError):
            spg.spg_lattice_site_map(*args)
    from paper_2502_02317_gb300 import _binding as b
    assert spg.lib.spg_lattice_site_map(3, 3, 0, None, None, None) == b.SPG_EINVAL


def test_binding_rejects_misread_tensors_before_any_launch():
    """Tensors the C ABI would misread (wrong dtype, not contiguous, not on
    a CUDA device) are refused by the binding before the library is called;
    these checks need no GPU."""
    import torch
    import paper_2502_02317_gb300 as spg
    from paper_2502_02317_gb300 import _binding as b
    bad = [torch.zeros((8, 8), dtype=torch.float32),            # wrong dtype
           torch.zeros((8, 8), dtype=torch.float64),            # host memory
           torch.zeros((8, 16), dtype=torch.float64)[:, ::2]]   # strided
    for t in bad:
        with pytest.raises(ValueError):
            spg.spg_truncate_static(t, 4)
        with pytest.raises(ValueError):
            b._device_tensor(t, torch.float64, "M")
    with pytest.raises(ValueError):
        b._device_tensor(torch.zeros(8, dtype=torch.float64), torch.float64, "M")
    assert b._stream_handle(None) is None
    assert b._stream_handle(0) is None
    assert b._stream_handle(1234).value == 1234


def test_autotuner_modes_on_the_host():
    """The autotuner's process-wide mode: on by default, every documented
    mode accepted, out-of-range ones refused; no shape is timed without a
    launch, and the report and clear calls need no device."""
    import paper_2502_02317_gb300 as spg
    prev = spg.spg_autotune_set(spg.SPG_TUNE_OFF)
    try:
        assert prev == spg.SPG_TUNE_ON
        last = spg.SPG_TUNE_OFF
        for mode in [spg.SPG_TUNE_ON] + [spg.SPG_TUNE_FORCE + k for k in range(4)]:
            assert spg.spg_autotune_set(mode) == last
            last = mode
        for bad in (-1, spg.SPG_TUNE_FORCE + 4):
            with pytest.raises(spg.SpgError) as e:
                spg.spg_autotune_set(bad)
            assert e.value.code == spg.SPG_EINVAL
        spg.spg_autotune_clear()
        assert spg.spg_autotune_report() == []
        n = ctypes.c_int32(-1)
        assert spg.lib.spg_autotune_report(ctypes.byref(n), None, 0) == 0 and n.value == 0
    finally:
        spg.spg_autotune_set(spg.SPG_TUNE_ON)
