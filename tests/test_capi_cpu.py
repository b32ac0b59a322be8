"""CPU-only checks of the C ABI: the library loads, exports every symbol that
include/fbcorr.h declares, validates arguments before touching a GPU, and its
generated kernel sources compile for sm_103a (NVRTC needs no GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_0911_3456_gb300 import _capi as C
from paper_0911_3456_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return C.load()


def header_functions():
    text = open(os.path.join(ROOT, "include", "fbcorr.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fbcorr_[a-z_0-9]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    names = header_functions()
    assert len(names) >= 19
    out = subprocess.run(["nm", "-D", "--defined-only", C.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (fbcorr_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert hasattr(lib, n)
    # the binding declares the same names
    assert set(C.PROTOTYPES) == set(names)


def test_version_and_status_strings(lib):
    assert b"sm_103a" in lib.fbcorr_version()
    for code, name in C.STATUS_NAMES.items():
        assert lib.fbcorr_status_string(code).decode() == name


def _create(lib, ins, fs, dtype=0, clamp=None):
    h = ctypes.c_void_p()
    st = lib.fbcorr_plan_create(ctypes.byref(h), C.I64_3(*ins), C.I64_4(*fs), dtype, C.epilogue(clamp))
    return st, h


@pytest.mark.parametrize("ins,fs,expect", [
    ((8, 8, 2), (1, 9, 3, 2), 2),          # fh > H
    ((8, 8, 2), (1, 3, 3, 4), 2),          # depth mismatch
    ((0, 8, 2), (1, 3, 3, 2), 2),          # zero dim
    ((8, 8, 2), (-1, 3, 3, 2), 2),         # negative dim
    ((70000, 70000, 1), (1, 1, 1, 1), 2),  # int32 overflow of H*W*D
    ((8, 8, 2), (1, 3, 3, 2), 2),          # placeholder replaced below
])
def test_plan_create_rejects_bad_shapes(lib, ins, fs, expect):
    if ins == (8, 8, 2) and fs == (1, 3, 3, 2):
        st, _ = _create(lib, ins, fs, dtype=7)
        assert st == 1  # bad dtype
        return
    st, h = _create(lib, ins, fs)
    assert st == expect, C.last_error()
    assert not h.value


def test_plan_create_rejects_bad_epilogue(lib):
    st, _ = _create(lib, (8, 8, 2), (1, 3, 3, 2), clamp=(1.0, 0.0))
    assert st == 1
    h = ctypes.c_void_p()
    st = lib.fbcorr_plan_create(ctypes.byref(h), C.I64_3(8, 8, 2), C.I64_4(1, 3, 3, 2), 0,
                                C.Epilogue(5, 0.0, 1.0))
    assert st == 1
    assert lib.fbcorr_plan_create(None, C.I64_3(8, 8, 2), C.I64_4(1, 3, 3, 2), 0, C.epilogue()) == 1


def test_null_plan_calls_fail_cleanly(lib):
    assert lib.fbcorr_forward(None, None, None, None, None, 0, None) == 1
    assert lib.fbcorr_backward(None, None, None, None, None, None, None, None, 0, None) == 1
    assert lib.fbcorr_plan_out_shape(None, C.I64_3()) == 1
    assert lib.fbcorr_plan_destroy(None) == 0
    assert lib.fbcorr_autotune(None, None) == 1


def test_valid_plan_without_gpu_reports_cuda_error(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    st, h = _create(lib, (16, 16, 4), (2, 3, 3, 4))
    assert st == 6 and "cuda" in C.last_error().lower() or st == 6


SHAPES = [
    ((128, 128, 8), (16, 9, 9, 8), None),
    ((256, 256, 8), (64, 9, 9, 8), (0.0, 1.0)),
    ((512, 512, 32), (256, 5, 5, 32), None),
    ((256, 256, 16), (64, 7, 7, 16), None),
    ((12, 12, 2), (3, 3, 3, 2), None),
    ((37, 45, 3), (5, 4, 2, 3), (-0.5, 0.5)),   # odd everything, fh != fw
    ((64, 64, 4), (16, 11, 11, 4), None),
    ((512, 512, 4), (32, 13, 13, 4), None),      # the paper's second table row
    ((128, 96, 8), (4, 8, 8, 8), None),          # even filter size
]


@pytest.mark.parametrize("ins,fs,clamp", SHAPES)
def test_generated_sources_compile(lib, ins, fs, clamp):
    log = ctypes.create_string_buffer(1 << 16)
    st = lib.fbcorr_rtcg_check(C.I64_3(*ins), C.I64_4(*fs), C.epilogue(clamp), b"heuristic", log,
                               len(log))
    assert st == 0, C.last_error() + log.value.decode()


@pytest.mark.parametrize("spec", [b"direct:tr=8,tf=8,wr=1,wf=2", b"direct:tr=2,tf=4,wr=4,wf=1",
                                  b"direct:tr=4,tf=8,wr=2,wf=4", b"direct:tr=8,tf=8,wr=2,wf=2,cc=4,pk=1",
                                  b"direct:tr=2,tf=4,wr=4,wf=1,cc=0,pk=1"])
def test_explicit_tile_specs_compile(lib, spec):
    log = ctypes.create_string_buffer(1 << 16)
    st = lib.fbcorr_rtcg_check(C.I64_3(64, 80, 8), C.I64_4(24, 5, 3, 8), C.epilogue((0, 1)), spec,
                               log, len(log))
    assert st == 0, C.last_error() + log.value.decode()
    st = lib.fbcorr_rtcg_check(C.I64_3(64, 80, 8), C.I64_4(24, 5, 3, 8), C.epilogue(), b"direct:bogus",
                               log, len(log))
    assert st == 1
    st = lib.fbcorr_rtcg_check(C.I64_3(64, 80, 8), C.I64_4(24, 5, 3, 8), C.epilogue(),
                               b"direct:tr=8,tf=8,wr=1,wf=2,cc=0,pk=2", log, len(log))
    assert st == 1


@pytest.mark.parametrize("spec,ok", [
    (b"direct:tr=8,tf=8,wr=1,wf=2,pk=1", True),          # pk without cc
    (b"direct:tr=8,tf=8,wr=1,wf=2,cc=4,pk=0", True),
    (b"direct:tr=8,tf=8,wr=1,wf=2,cc=4,pk=1x", False),   # trailing text
    (b"direct:tr=8,tf=8,wr=1,wf=2,cc=4,zz=1", False),    # unknown field
    (b"direct:tr=8,tf=8,wr=1,wf=2,pk=1,cc=4", False),    # fields out of order
    (b"direct:tr=8,tf=8,wr=1,wf=2 ", False),
    (b"direct:tr=8,tf=6,wr=1,wf=2", False),              # TF not a multiple of 4
    (b"direct:tr=4,tf=8,wr=2,wf=1,cc=0,pk=1,ks=8,wq=4", True),    # K-split tile
    (b"direct:tr=4,tf=8,wr=2,wf=1,ks=8,wq=4", True),
    (b"direct:tr=4,tf=8,wr=2,wf=1,cc=0,ks=8", False),             # ks needs wq
    (b"direct:tr=4,tf=8,wr=2,wf=1,cc=0,ks=6,wq=4", False),        # ks: 4, 8, 16 or 32
    (b"direct:tr=2,tf=4,wr=2,wf=1,cc=0,ks=8,wq=4", False),        # 4 pairs do not split over 8 lanes
    (b"direct:tr=4,tf=8,wr=2,wf=1,cc=4,ks=8,wq=4", False),        # K split stages the whole depth
    (b"direct:tr=4,tf=8,wr=2,wf=1,cc=0,ks=8,wq=4,pk=1", False),   # fields out of order
    (b"direct:tr=4,tf=8,wr=2,wf=1,cc=0,ks=1,wq=2", False),        # no split: one warp per 32 columns
    (b"direct:tr=16,tf=4,wr=1,wf=4,cc=0,pk=1,ks=8,wq=2,sh=1", True),   # share in the high lane bits
    (b"direct:tr=4,tf=8,wr=2,wf=1,cc=0,ks=8,wq=4,sh=2", False),
    (b"direct:tr=4,tf=8,wr=2,wf=1,cc=0,sh=1", False),              # sh only with a K split
    (b"direct:tr=8,tf=8,wr=2,wf=2,cc=8,pk=1,mb=2", True),          # two CTAs per SM (launch bounds)
    (b"direct:tr=8,tf=4,wr=3,wf=2,cc=0,pk=1,ks=8,wq=2,sh=1,mb=3", True),
    (b"direct:tr=8,tf=8,wr=2,wf=2,cc=8,pk=1,mb=1", False),         # mb: 2, 3 or 4
    (b"direct:tr=8,tf=8,wr=2,wf=2,cc=8,pk=1,mb=5", False),
    (b"direct:tr=8,tf=8,wr=2,wf=2,cc=8,mb=2,pk=1", False),         # fields out of order
])
def test_direct_spec_parsing_is_strict(lib, spec, ok):
    log = ctypes.create_string_buffer(1 << 16)
    st = lib.fbcorr_rtcg_check(C.I64_3(64, 80, 8), C.I64_4(24, 5, 3, 8), C.epilogue(), spec, log, len(log))
    assert (st == 0) == ok, (st, C.last_error())


@pytest.mark.parametrize("D,N,spec", [
    (8, 16, b"direct:tr=4,tf=8,wr=2,wf=1,cc=0,pk=1,ks=8,wq=4"),    # the first configuration's depth
    (8, 16, b"direct:tr=2,tf=16,wr=4,wf=1,cc=0,ks=16,wq=2"),       # eight padding channels per pixel
    (3, 5, b"direct:tr=4,tf=4,wr=1,wf=2,cc=0,pk=1,ks=4,wq=8"),     # depth 3 padded to 4, scalar staging
    (16, 12, b"direct:tr=8,tf=8,wr=1,wf=1,cc=0,ks=32,wq=2"),       # one column per warp
    (24, 20, b"direct:tr=4,tf=8,wr=2,wf=2,cc=0,pk=1,ks=8,wq=2"),   # three channels per lane
    (8, 16, b"direct:tr=16,tf=4,wr=1,wf=4,cc=0,pk=1,ks=8,wq=2,sh=1"),   # share in the high lane bits
])
def test_ksplit_tiles_compile(lib, D, N, spec):
    """The K-split forward tile compiles for sm_103a with the clamp epilogue;
    a backward (flipped) problem never takes it."""
    log = ctypes.create_string_buffer(1 << 16)
    st = lib.fbcorr_rtcg_check(C.I64_3(40, 50, D), C.I64_4(N, 5, 3, D), C.epilogue((-1, 1)), spec, log, len(log))
    assert st == 0, C.last_error() + log.value.decode()


@pytest.mark.parametrize("shape,clamp,spec,expect", [
    ((256, 256, 16, 64, 7, 7), None, b"direct:tr=7,tf=4,wr=2,wf=4,cc=4,pk=1,ks=4,wq=2", 0),
    ((256, 256, 16, 64, 7, 7), None, b"direct:tr=8,tf=4,wr=2,wf=4,cc=8,pk=1,pf=1,ks=4,wq=2", 0),
    ((40, 52, 16, 24, 7, 7), None, b"direct:tr=6,tf=8,wr=2,wf=2,cc=16,ks=8,wq=1", 0),
    ((61, 45, 4, 8, 5, 4), None, b"direct:tr=7,tf=4,wr=2,wf=4,cc=8,pk=1,ks=8,wq=2", 0),
    ((40, 52, 16, 24, 7, 7), (0, 1), b"direct:tr=7,tf=4,wr=2,wf=4,cc=4,pk=1,ks=4,wq=2", 3),   # clamp mask
    ((40, 52, 6, 24, 7, 7), None, b"direct:tr=7,tf=4,wr=2,wf=4,cc=4,pk=1,ks=4,wq=2", 3),      # D % 4
    ((40, 52, 16, 22, 7, 7), None, b"direct:tr=7,tf=4,wr=2,wf=4,cc=4,pk=1,ks=4,wq=2", 3),     # N % 4
    ((40, 52, 16, 24, 7, 7), None, b"direct:tr=7,tf=4,wr=2,wf=4,cc=6,pk=1,ks=4,wq=2", 1),     # cc % ks
    ((40, 52, 16, 24, 7, 7), None, b"direct:tr=7,tf=4,wr=2,wf=4,cc=40,pk=1,ks=8,wq=2", 1),    # 5 per lane
    ((40, 52, 16, 24, 7, 7), None, b"direct:tr=7,tf=4,wr=2,wf=4,cc=8,pk=1,ks=8,wq=2,sh=1", 1),
])
def test_chunked_ksplit_dx_tiles_compile(lib, shape, clamp, spec, expect):
    """The chunked K-split dL/dx tile compiles for sm_103a on the flipped
    problem; shapes whose dL/dx it cannot take and malformed specs are refused."""
    H, W, D, N, fh, fw = shape
    log = ctypes.create_string_buffer(1 << 16)
    st = lib.fbcorr_rtcg_check(C.I64_3(H, W, D), C.I64_4(N, fh, fw, D), C.epilogue(clamp), spec, log, len(log))
    assert st == expect, C.last_error() + log.value.decode()


@pytest.mark.parametrize("D,f,spec", [
    (32, 5, b"tcgen05:na=2,nb=4,nt=256,bt=5,ew=4,fz=1,nr=0,cw=4"),    # the precision workload, converters from registers
    (32, 5, b"tcgen05:na=3,nb=3,nt=256,bt=3,ew=8,fz=2,nr=3,cw=8"),    # raw-row ring; two stages, the second partial
    (8, 9, b"tcgen05:na=2,nb=4,nt=128,bt=2,ew=4,fz=1,nr=0,cw=8"),     # paper row 1 depth, odd last stage
    (48, 7, b"tcgen05:na=2,nb=4,nt=256,bt=4,ew=8,fz=2,nr=2,cw=8"),    # six chunk planes, raw-row ring
    (64, 13, b"tcgen05:na=2,nb=2,nt=256,bt=1,ew=4,fz=0,nr=0,cw=0"),   # the deepest supported depth, pre-pass
    (32, 5, b"tcgen05:na=3,nb=2,nt=256,bt=5,ew=8,fz=1,nr=0,cw=8,ts=32,sb=1"),       # tiled bulk stores
    (16, 3, b"tcgen05:na=3,nb=4,nt=256,bt=2,ew=8,fz=2,nr=2,cw=8,ts=1,sb=1"),        # staged stores
    (32, 5, b"tcgen05:na=2,nb=3,nt=256,bt=1,ew=4,fz=1,nr=0,cw=4,ts=32,sb=3"),       # three staging slots
    (32, 5, b"tcgen05:na=2,nb=5,nt=128,bt=5,ew=4,fz=1,nr=0,cw=8,rs=1"),             # resident bank
    (16, 3, b"tcgen05:na=3,nb=3,nt=256,bt=3,ew=8,fz=2,nr=2,cw=8,ts=1,sb=1,rs=1"),   # resident, staged stores
    (32, 5, b"tcgen05:na=2,nb=8,nt=256,bt=1,ew=4,fz=1,nr=0,cw=8,ts=32,sb=1,cg=2"),  # CTA pair, tiled stores
    (32, 5, b"tcgen05:na=3,nb=6,nt=256,bt=3,ew=8,fz=2,nr=3,cw=8,cg=2"),             # CTA pair, raw-row ring
    (32, 5, b"tcgen05:na=6,nb=3,nt=256,bt=2,ew=4,fz=2,nr=3,cw=8,ts=32,sb=1,sw=1"),  # sliding window, raw ring
    (16, 7, b"tcgen05:na=7,nb=3,nt=256,bt=3,ew=8,fz=1,nr=0,cw=8,sw=1"),             # sliding window, registers
    (16, 3, b"tcgen05:na=3,nb=4,nt=256,bt=2,ew=8,fz=0,nr=0,cw=0,ts=1,sb=1,cg=2"),   # CTA pair, pre-pass, staged
])
def test_tensor_core_kernels_compile(lib, D, f, spec):
    """The run-time generated tcgen05 kernel of a spec compiles for sm_103a in
    BF16 and split-BF16 form (filter width and taps per stage baked in)."""
    log = ctypes.create_string_buffer(1 << 16)
    st = lib.fbcorr_rtcg_check(C.I64_3(64, 64, D), C.I64_4(16, f, f, D), C.epilogue(), spec, log, len(log))
    assert st == 0, C.last_error() + log.value.decode()


@pytest.mark.parametrize("D,f,spec,status", [
    (48, 7, b"tcgen05:na=2,nb=4,nt=256,bt=2,ew=4,fz=1,nr=0,cw=8", 3),   # register conversion needs D <= 32
    (30, 7, b"tcgen05:na=2,nb=4,nt=256,bt=2,ew=4,fz=2,nr=2,cw=8", 3),   # in-kernel conversion needs D % 4 == 0
    (32, 3, b"tcgen05:na=2,nb=4,nt=256,bt=4,ew=4,fz=0,nr=0,cw=0", 3),   # more taps per stage than fw
    (32, 5, b"tcgen05:na=2,nb=4,nt=256,bt=2,ew=6,fz=0,nr=0,cw=0", 1),   # epilogue warps must be 4 or 8
    (32, 5, b"tcgen05:na=2,nb=4,nt=256,bt=2,ew=4,fz=0", 1),        # missing field: not a spec of this kernel
    (32, 5, b"tcgen05:na=2,nb=4,nt=256,bt=2,ew=4,fz=2,nr=0,cw=8", 1),   # the raw ring needs slots
    (32, 5, b"tcgen05:na=2,nb=4,nt=256,bt=2,ew=4,fz=1,nr=0,cw=0", 1),   # in-kernel conversion needs converter warps
    (32, 5, b"tcgen05:na=2,nb=4,nt=256,bt=2,ew=8,fz=1,nr=0,cw=8,ts=2,sb=1", 1),    # store modes: 1 or 32
    (32, 5, b"tcgen05:na=2,nb=4,nt=256,bt=2,ew=8,fz=1,nr=0,cw=8,ts=32,sb=4", 1),   # at most three staging slots
    (32, 5, b"tcgen05:na=2,nb=4,nt=256,bt=2,ew=8,fz=1,nr=0,cw=8,ts=1,sb=2", 1),    # the staged path has one slot
    (32, 5, b"tcgen05:na=2,nb=4,nt=256,bt=2,ew=8,fz=1,nr=0,cw=8,sb=1,ts=1", 1),    # suffix fields in order
    (32, 5, b"tcgen05:na=2,nb=4,nt=256,bt=2,ew=8,fz=1,nr=0,cw=8,ts=1,sb=1,", 1),   # nothing after the suffix
    (32, 5, b"tcgen05:na=2,nb=5,nt=128,bt=5,ew=4,fz=1,nr=0,cw=8,rs=2", 1),          # rs=1 only
    (32, 5, b"tcgen05:na=2,nb=5,nt=128,bt=5,ew=8,fz=1,nr=0,cw=8,rs=1,ts=1,sb=1", 1),   # stores before rs
    (32, 5, b"tcgen05:na=2,nb=5,nt=256,bt=5,ew=4,fz=1,nr=0,cw=8,cg=1", 1),          # cg=2 only
    (32, 5, b"tcgen05:na=2,nb=5,nt=256,bt=5,ew=4,fz=1,nr=0,cw=8,cg=2,rs=1", 1),     # rs before cg
    (32, 5, b"tcgen05:na=2,nb=5,nt=256,bt=5,ew=4,fz=1,nr=0,cw=8,rs=1,cg=2", 1),     # a pair streams the bank
    (32, 5, b"tcgen05:na=6,nb=3,nt=256,bt=2,ew=4,fz=1,nr=0,cw=8,sw=2", 1),          # sw=1 only
    (32, 5, b"tcgen05:na=6,nb=3,nt=256,bt=2,ew=4,fz=1,nr=0,cw=8,cg=2,sw=1", 1),     # the window runs single CTAs
    (32, 5, b"tcgen05:na=6,nb=3,nt=128,bt=2,ew=4,fz=1,nr=0,cw=8,rs=1,sw=1", 1),     # and a streamed bank
    (32, 5, b"tcgen05:na=6,nb=3,nt=256,bt=2,ew=4,fz=1,nr=0,cw=8,sw=1,ts=1,sb=1", 1),   # stores before sw
])
def test_tensor_core_spec_refusals(lib, D, f, spec, status):
    log = ctypes.create_string_buffer(1 << 16)
    st = lib.fbcorr_rtcg_check(C.I64_3(64, 64, D), C.I64_4(16, f, f, D), C.epilogue(), spec, log, len(log))
    assert st == status, C.last_error()


def test_nvrtc_fault_injection_reports_nvrtc_error():
    """FBCORR_FAULT=nvrtc makes code generation fail; the status says so."""
    code = ("import ctypes\nfrom paper_0911_3456_gb300 import _capi as C\nlib=C.load()\n"
            "log=ctypes.create_string_buffer(4096)\n"
            "print(lib.fbcorr_rtcg_check(C.I64_3(16,16,4), C.I64_4(2,3,3,4), C.epilogue(), b'heuristic', log, 4096))\n")
    env = dict(os.environ, FBCORR_FAULT="nvrtc")
    r = subprocess.run(["python", "-c", code], capture_output=True, text=True, env=env, cwd=ROOT)
    assert r.stdout.strip().splitlines()[-1] == "7", r.stderr


@pytest.mark.parametrize("ks", ["0", "1"])
def test_batch_kernel_source_compiles(lib, ks, monkeypatch):
    """The single persistent kernel of a batch plan (several filter sizes and
    depths in one switch) compiles for sm_103a, also with K-split tiles in the
    variants that take one (FBCORR_BATCH_KS=1)."""
    monkeypatch.setenv("FBCORR_BATCH_KS", ks)
    shapes = [(40, 70, 8, 16, 3, 3), (33, 45, 4, 32, 5, 5), (20, 150, 32, 64, 11, 11),
              (17, 19, 3, 5, 2, 4)]
    n = len(shapes)
    ins = (ctypes.c_int64 * (3 * n))(*[v for (H, W, D, N, fh, fw) in shapes for v in (H, W, D)])
    fls = (ctypes.c_int64 * (4 * n))(*[v for (H, W, D, N, fh, fw) in shapes for v in (N, fh, fw, D)])
    log = ctypes.create_string_buffer(1 << 16)
    st = lib.fbcorr_batch_rtcg_check(n, ins, fls, C.epilogue((0.0, 1.0)), log, len(log))
    assert st == 0, C.last_error() + log.value.decode()


@pytest.mark.parametrize("dtype", [0, 1, 2])
@pytest.mark.parametrize("expr", [b"y > 0.f ? y : lo * y", b"tanhf(y) * hi + 0.5f * (float)(n % 3)",
                                  b"fminf(fmaxf(y, lo), hi)"])
def test_snippet_epilogue_compiles(lib, dtype, expr):
    """A user expression becomes the store epilogue of the generated forward
    kernel (FP32 direct tile or tcgen05), compiled by NVRTC without a GPU."""
    log = ctypes.create_string_buffer(1 << 16)
    st = lib.fbcorr_snippet_check(C.I64_3(40, 52, 16), C.I64_4(12, 5, 3, 16), dtype, expr, log, len(log))
    assert st == 0, C.last_error() + log.value.decode()


@pytest.mark.parametrize("expr,status", [
    (b"y +", 7),                  # does not compile: NVRTC error, with the log
    (b"y; y = 0.f", 1),           # statements are refused before compiling
    (b"{ return y; }", 1),
    (b"", 1),
    (b"y * \"1\"", 1),
])
def test_snippet_epilogue_refusals(lib, expr, status):
    log = ctypes.create_string_buffer(1 << 16)
    st = lib.fbcorr_snippet_check(C.I64_3(40, 52, 16), C.I64_4(12, 5, 3, 16), 0, expr, log, len(log))
    assert st == status, C.last_error()
    if status == 7:
        assert b"error" in log.value


def test_snippet_kind_needs_its_own_entry_points(lib):
    """A SNIPPET epilogue kind is refused by the clamp-style checks and by batch plans."""
    log = ctypes.create_string_buffer(1 << 12)
    epi = C.Epilogue(C.EPI_SNIPPET, 0.0, 0.0)
    assert lib.fbcorr_rtcg_check(C.I64_3(16, 16, 4), C.I64_4(2, 3, 3, 4), epi, b"heuristic", log, len(log)) == 1
    ins = (ctypes.c_int64 * 3)(16, 16, 4)
    fls = (ctypes.c_int64 * 4)(2, 3, 3, 4)
    assert lib.fbcorr_batch_rtcg_check(1, ins, fls, epi, log, len(log)) == 3


def test_fma_probe_rejects_bad_arguments_before_any_launch(lib):
    t = ctypes.c_double()
    assert lib.fbcorr_fp32_fma_probe(0, 0, ctypes.byref(t), None) == 1
    assert lib.fbcorr_fp32_fma_probe(2, 100, ctypes.byref(t), None) == 1
    assert lib.fbcorr_fp32_fma_probe(0, (1 << 24) + 1, ctypes.byref(t), None) == 1
    assert lib.fbcorr_fp32_fma_probe(1, 100, None, None) == 1
    assert "iters" in C.last_error()
