"""The C-ABI library builds, loads and exports every symbol include/bls.h declares; the
ctypes structs match the C layout; argument checks that need no GPU behave."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_1112_1701_b300 import bls, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bls.h")


@pytest.fixture(scope="module")
def L():
    build.build()
    return bls.lib()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bls_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("bls_plan_create", "bls_search", "bls_submit", "bls_poll",
                     "bls_plan_destroy", "bls_last_error"):
        assert required in names
    assert set(names) == set(bls.EXPORTS)


def test_library_exports_every_declared_symbol(L):
    out = subprocess.run(["nm", "-D", "--defined-only", bls.LIB_PATH], check=True,
                         capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (bls_[a-z_]+)", out))
    for name in declared_functions():
        assert name in exported, name
        assert hasattr(L, name)


def test_debug_library_exports_the_same_symbols(L):
    """libbls_debug.so (device-side index checks, loaded with BLS_DEBUG=1) is built beside
    libbls.so from the same sources and exports the same boundary."""
    path = os.path.join(os.path.dirname(bls.LIB_PATH), "libbls_debug.so")
    out = subprocess.run(["nm", "-D", "--defined-only", path], check=True,
                         capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (bls_[a-z_]+)", out))
    assert set(declared_functions()) <= exported


def test_struct_layout_matches_c(tmp_path):
    prog = tmp_path / "sz.c"
    prog.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "bls.h"\n'
        'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(bls_plan_desc),'
        ' sizeof(bls_curve), sizeof(bls_peak), sizeof(bls_server_stats),'
        ' offsetof(bls_peak, freq), offsetof(bls_curve, nb), sizeof(bls_window_desc),'
        ' offsetof(bls_window_desc, duration), sizeof(bls_profile), sizeof(bls_shape),'
        ' sizeof(bls_shape_grid), sizeof(bls_var_desc), sizeof(bls_var_star)); return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)],
                   check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                           check=True).stdout.split()]
    assert vals == [C.sizeof(bls.PlanDesc), C.sizeof(bls.CurveStruct),
                    C.sizeof(bls.PeakStruct), C.sizeof(bls.ServerStats),
                    bls.PeakStruct.freq.offset, bls.CurveStruct.nb.offset,
                    C.sizeof(bls.WindowDesc), bls.WindowDesc.duration.offset,
                    C.sizeof(bls.Profile), bls.SHAPE_DTYPE.itemsize, C.sizeof(bls.ShapeGrid),
                    C.sizeof(bls.VarDesc), bls.VAR_DTYPE.itemsize]


def test_kminmax_matches_reading(L):
    assert bls.kminmax(100, 0.01, 0.10) == (1, 10)
    assert bls.kminmax(200, 0.005, 0.15) == (1, 30)
    assert bls.kminmax(256, 0.005, 0.15) == (1, 39)
    with pytest.raises(bls.BLSError) as ei:
        bls.kminmax(1, 0.1, 0.2)
    assert ei.value.status == bls.ERR_INVALID


def test_kminmax_agrees_with_oracle(L):
    import oracle
    for nb in (2, 3, 10, 57, 100, 200, 256, 400, 1000):
        for q0, q1 in ((0.001, 0.01), (0.005, 0.15), (0.01, 0.1), (0.3, 0.9), (0.05, 0.05)):
            assert bls.kminmax(nb, q0, q1) == oracle.kminmax(nb, q0, q1)


def test_plan_rejects_bad_descriptors_before_touching_cuda(L):
    for kw in (dict(nb=1), dict(topk=0), dict(topk=99), dict(qmin=0.2, qmax=0.1),
               dict(freqs_per_block=17), dict(kmin=5, kmax=2)):
        with pytest.raises(bls.BLSError) as ei:
            bls.Plan(**kw)
        assert ei.value.status == bls.ERR_INVALID
        assert bls.lib().bls_last_error()


def test_packed_curves_descriptors():
    """PackedCurves writes the same bls_curve descriptors as one CurveInput per curve
    (pointers at each curve's offset into the packed arrays)."""
    import numpy as np
    from paper_1112_1701_b300 import synth
    b = synth.config2(ncurves=5, nf=100, seed=4)
    pc = bls.packed_from_batch(b)
    t, y, dy = pc.keep
    keep = []
    ref = [bls._struct(ci, keep) for ci in bls.curves_from_batch(b)]
    o = 0
    for k, c in enumerate(b.curves):
        a, r = pc.arr[k], ref[k]
        for f, _ in bls.CurveStruct._fields_:
            if f not in ("t", "y", "dy"):
                assert (getattr(a, f) or 0) == (getattr(r, f) or 0), (k, f)
        assert (a.t, a.y, a.dy) == (t.ctypes.data + 8 * o, y.ctypes.data + 4 * o,
                                    dy.ctypes.data + 4 * o)
        o += len(c.t)
    assert len(pc) == 5 and pc.total_nf == 500
    with pytest.raises(ValueError):
        bls.PackedCurves(t[:10], y, dy, [len(c.t) for c in b.curves], 100, 0.1, 0.01)


def test_packed_curves_without_errors_and_scalar_grids():
    """dy = None packs as NULL (unit weights); scalar grid fields apply to every curve."""
    import numpy as np
    t = np.linspace(0.0, 10.0, 30)
    y = np.ones(30, np.float32)
    pc = bls.PackedCurves(t, y, None, [10, 20], 500, 0.2, 0.001, nb=150, qmin=0.01, qmax=0.1)
    assert [pc.arr[k].dy for k in range(2)] == [None, None]
    assert [pc.arr[k].n for k in range(2)] == [10, 20]
    assert pc.arr[1].t == t.ctypes.data + 8 * 10 and pc.arr[1].y == y.ctypes.data + 4 * 10
    assert all(pc.arr[k].nf == 500 and pc.arr[k].nb == 150 for k in range(2))
    assert pc.total_nf == 1000


def test_binding_rejects_mistyped_and_short_tensors():
    """Tensors are passed to the library by address, so the binding checks their dtype,
    contiguity and length first (no GPU needed: CPU tensors take the same checks)."""
    torch = pytest.importorskip("torch")
    t = torch.linspace(0, 10, 50, dtype=torch.float64)
    y = torch.ones(50, dtype=torch.float32)
    cases = [
        bls.CurveInput(t.float(), y, None, nf=5, fmin=0.1, df=0.1),          # t not FP64
        bls.CurveInput(t, y.double(), None, nf=5, fmin=0.1, df=0.1),         # y not FP32
        bls.CurveInput(t, y, y.double(), nf=5, fmin=0.1, df=0.1),            # dy not FP32
        bls.CurveInput(t, y[:40], None, nf=5, fmin=0.1, df=0.1),             # y short
        bls.CurveInput(t, y, y[:49], nf=5, fmin=0.1, df=0.1),                # dy short
        bls.CurveInput(t[::2], y[:25], None, nf=5, fmin=0.1, df=0.1),        # not contiguous
        bls.CurveInput(t, y, None, freqs=torch.ones(5, dtype=torch.float32)),  # freqs FP32
    ]
    for c in cases:
        with pytest.raises(bls.BLSError) as ei:
            bls._struct(c, [])
        assert ei.value.status == bls.ERR_INVALID
    import numpy as np
    with pytest.raises(bls.BLSError):                                      # numpy, y short
        bls._struct(bls.CurveInput(np.zeros(5), np.zeros(4, np.float32), None, nf=2), [])
    ok = bls._struct(bls.CurveInput(t, y, None, nf=5, fmin=0.1, df=0.1), [])
    assert ok.n == 50 and ok.nf == 5


def test_static_search_checks_output_sizes_before_the_call():
    """bls_search_static cannot see the size of a device buffer: the binding refuses
    outputs smaller than what the call writes (topk records, nf spectrum values)."""
    torch = pytest.importorskip("torch")
    t = torch.linspace(0, 10, 50, dtype=torch.float64)
    c = bls.CurveInput(t, torch.ones(50, dtype=torch.float32), None, nf=10, fmin=0.1, df=0.1,
                       nb=20, qmin=0.05, qmax=0.2)
    one = torch.zeros(bls.PEAK_DTYPE.itemsize, dtype=torch.uint8)
    for kw in (dict(topk=2, peaks=one), dict(peaks=None),
               dict(peaks=one, spectrum=torch.zeros(9, dtype=torch.float32)),
               dict(peaks=one, spectrum=torch.zeros(10, dtype=torch.float64))):
        with pytest.raises(bls.BLSError) as ei:
            bls.search_static(c, **kw)
        assert ei.value.status == bls.ERR_INVALID
