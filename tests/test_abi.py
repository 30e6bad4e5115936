"""The C ABI without a GPU: the library loads, exports every entry point the
header declares, and rejects bad arguments before touching the device."""
import os
import re

import numpy as np
import pytest

from paper_2208_09822_gb300 import build as B
from paper_2208_09822_gb300 import iaat
from paper_2208_09822_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    B.build()
    return iaat.lib()


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "iaat.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(iaat_[a-z0-9_]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert "iaat_gemm_grouped" in names and "iaat_plan_create" in names
    for n in names:
        assert hasattr(L, n), n


def test_version(L):
    assert "sm_103a" in iaat.iaat_version()


def _desc(**kw):
    d = np.zeros(1, iaat.DESC_DTYPE)
    base = dict(M=4, N=4, K=4, lda=4, ldb=4, ldc=4, transA=0, transB=0, alpha=1.0, beta=0.0,
                A=0x10000, B=0x20000, C=0x30000)
    base.update(kw)
    for k, v in base.items():
        d[k] = v
    return d


@pytest.mark.parametrize("kw,status", [
    (dict(M=-1), 1), (dict(lda=3), 1), (dict(ldb=3), 1), (dict(ldc=3), 1),
    (dict(transA=2), 1), (dict(C=0), 1), (dict(A=0), 1),
    (dict(M=80, N=80, K=81, lda=80, ldb=81, ldc=80), 2),                     # 518400 > 512000
    (dict(M=32, N=32, K=33, transA=1, lda=33, ldb=33, ldc=32), 2),          # TN: 33792 > 32768
    (dict(A=0x10002), 3), (dict(C=0x30001), 3),
])
def test_plan_create_rejects(L, kw, status):
    with pytest.raises(iaat.IaatError) as e:
        iaat.iaat_plan_create(_desc(**kw), iaat.IAAT_F32)
    assert e.value.status == status
    assert "instance 0" in e.value.message


def test_domain_boundary_is_inclusive(L):
    """cbrt(MNK) <= 80 (Sec. I): 80^3 itself is small; TN's bound is 32^3."""
    rows = [l.split() for l in open(os.path.join(ROOT, "tests", "golden", "domain_bounds.txt"))
            if l.strip() and not l.startswith("#")]
    lim = {c: int(v) ** 3 for c, v in rows}
    assert lim["NN"] == 512000 and lim["TN"] == 32768
    assert W.in_domain(80, 80, 80, 0, 0) and not W.in_domain(80, 80, 81, 0, 0)
    assert W.in_domain(32, 32, 32, 1, 0) and not W.in_domain(32, 32, 33, 1, 0)
    assert W.in_domain(32, 32, 33, 1, 1)   # TT keeps the larger bound


@pytest.mark.parametrize("K", [20000, 40000])
def test_plan_create_rejects_unstageable_k(L, K):
    """1 x 1 x K is small (MNK <= 512000) but a row of A and a column of B
    that long do not fit one pipeline stage of the stage-program kernels
    (tensor-core or CUDA-core), and those never cut K: a plan on them alone
    (kernel = 1) is rejected with UNSUPPORTED, before any device work.  (A
    default tensor-core plan sends such an instance to the warp-tile kernel,
    which stages K in pieces; the GPU tests cover that.)"""
    for prec, kernel in ((1, 1), (0, 1)):
        with pytest.raises(iaat.IaatError) as e:
            iaat.iaat_plan_create(_desc(M=1, N=1, K=K, lda=1, ldb=K, ldc=1), iaat.IAAT_F32, prec, kernel=kernel)
        assert e.value.status == 4
        assert "instance 0" in e.value.message


@pytest.mark.parametrize("prec", [iaat.IAAT_PREC_3XBF16, iaat.IAAT_PREC_6XBF16])
def test_fp64_rejects_tensor_precisions(L, prec):
    with pytest.raises(iaat.IaatError) as e:
        iaat.iaat_plan_create(_desc(), iaat.IAAT_F64, prec)
    assert e.value.status == 4


@pytest.mark.parametrize("prec", [-1, 5])
def test_unknown_precision_is_rejected(L, prec):
    with pytest.raises(iaat.IaatError) as e:
        iaat.iaat_plan_create(_desc(), iaat.IAAT_F32, prec)
    assert e.value.status == 1


def test_single_call_rejects(L):
    with pytest.raises(iaat.IaatError) as e:
        iaat.iaat_sgemm(0, 0, 81, 80, 80, 1.0, 0x1000, 81, 0x2000, 80, 0.0, 0x3000, 81)
    assert e.value.status == 2
    with pytest.raises(iaat.IaatError) as e:
        iaat.iaat_dgemm(0, 0, 4, 4, 4, 1.0, 0x1004, 4, 0x2000, 4, 0.0, 0x3000, 4)
    assert e.value.status == 3


def test_quick_returns_touch_nothing(L):
    # M == 0 / N == 0 is a no-op with any pointers; alpha == 0 with beta == 1 too
    iaat.iaat_sgemm(0, 0, 0, 5, 5, 1.0, 0, 1, 0, 5, 0.0, 0, 1)
    iaat.iaat_sgemm(0, 0, 5, 0, 5, 1.0, 0, 5, 0, 5, 0.0, 0, 5)
    iaat.iaat_sgemm(0, 0, 5, 5, 5, 0.0, 0, 5, 0, 5, 1.0, 0x3000, 5)


def _cdesc(**kw):
    d = np.zeros(1, iaat.CDESC_DTYPE)
    base = dict(M=4, N=4, K=4, lda=4, ldb=4, ldc=4, transA=0, transB=0, alpha_re=1.0, alpha_im=0.5,
                beta_re=0.0, beta_im=0.0, A=0x10000, B=0x20000, C=0x30000)
    base.update(kw)
    for k, v in base.items():
        d[k] = v
    return d


@pytest.mark.parametrize("dtype", [iaat.IAAT_C32, iaat.IAAT_C64])
@pytest.mark.parametrize("kw,status", [
    (dict(M=-1), 1), (dict(lda=3), 1), (dict(ldc=3), 1), (dict(transB=2), 1), (dict(C=0), 1),
    (dict(M=80, N=80, K=81, lda=80, ldb=81, ldc=80), 2),
    (dict(M=32, N=32, K=33, transA=1, lda=33, ldb=33, ldc=32), 2),
    (dict(A=0x10004), 3),
])
def test_complex_plan_create_rejects(L, dtype, kw, status):
    with pytest.raises(iaat.IaatError) as e:
        iaat.iaat_plan_create_complex(_cdesc(**kw), dtype)
    assert e.value.status == status
    assert "instance 0" in e.value.message


def test_complex_alignment_is_the_element_size(L):
    """A pointer 8 bytes past a 16-byte boundary is aligned for complex float
    but not for complex double (elements of 8 and 16 bytes)."""
    with pytest.raises(iaat.IaatError) as e:
        iaat.iaat_plan_create_complex(_cdesc(C=0x30008), iaat.IAAT_C64)
    assert e.value.status == 3
    with pytest.raises(iaat.IaatError) as e:   # passes the alignment check, fails the next one
        iaat.iaat_plan_create_complex(_cdesc(C=0x30008, ldc=3), iaat.IAAT_C32)
    assert e.value.status == 1


def test_complex_dtypes_have_their_own_entry(L):
    """iaat_plan_create refuses complex dtypes; iaat_plan_create_complex
    refuses real ones."""
    for dt in (iaat.IAAT_C32, iaat.IAAT_C64, 4):
        with pytest.raises(iaat.IaatError) as e:
            iaat.iaat_plan_create(_desc(), dt)
        assert e.value.status == 1
    for dt in (iaat.IAAT_F32, iaat.IAAT_F64, -1, 4):
        with pytest.raises(iaat.IaatError) as e:
            iaat.iaat_plan_create_complex(_cdesc(), dt)
        assert e.value.status == 1


def test_complex_tiler_uses_the_complex_family():
    """The host tiler covers C exactly for every dtype; complex double tiles
    are at most 32 x 16 or 16 x 32 (its register-tile family), and a
    one-column C takes one-column tiles (no idle lane columns)."""
    for dt in (iaat.IAAT_C32, iaat.IAAT_C64):
        for M, N, K in [(1, 1, 1), (15, 15, 15), (33, 17, 9), (80, 80, 80), (64, 5, 80)]:
            blocks = iaat.iaat_tile(dt, 0, 0, M, N, K)
            cover = np.zeros((M, N), int)
            for r0, c0, h, w in blocks:
                cover[r0:r0 + h, c0:c0 + w] += 1
                if dt == iaat.IAAT_C64:
                    assert h * w <= 512, (M, N, K, h, w)
            assert (cover == 1).all(), (dt, M, N, K)
    assert all(w == 1 for _, _, _, w in iaat.iaat_tile(iaat.IAAT_C64, 0, 0, 32, 1, 40))
    with pytest.raises(iaat.IaatError) as e:
        iaat.iaat_plan_create_complex(_cdesc(), iaat.IAAT_C32, force_variant=6)
    assert e.value.status == 1


def test_routed_plan_validates_with_caller_indices(L):
    """A routed tensor-core plan checks every instance before splitting, so
    the error names the caller's index; a negative threshold is refused."""
    d = np.concatenate([_desc(K=2), _desc(K=20, ldb=20), _desc(K=3), _desc(K=30, ldb=30, ldc=3)])
    with pytest.raises(iaat.IaatError) as e:
        iaat.iaat_plan_create(d, iaat.IAAT_F32, iaat.IAAT_PREC_3XBF16, route_k_below=8)
    assert e.value.status == 1 and "instance 3" in e.value.message
    with pytest.raises(iaat.IaatError) as e:
        iaat.iaat_plan_create(_desc(), iaat.IAAT_F32, iaat.IAAT_PREC_3XBF16, route_k_below=-1)
    assert e.value.status == 1
    with pytest.raises(iaat.IaatError) as e:
        iaat.iaat_plan_create(_desc(), iaat.IAAT_F32, iaat.IAAT_PREC_3XBF16, route_mnk_below=-1)
    assert e.value.status == 1 and "route_mnk_below" in e.value.message
    # routing by size alone (route_k_below 0) also validates with the caller's index
    with pytest.raises(iaat.IaatError) as e:
        iaat.iaat_plan_create(d, iaat.IAAT_F32, iaat.IAAT_PREC_3XBF16, route_mnk_below=4096)
    assert e.value.status == 1 and "instance 3" in e.value.message
    # the routed part's kernel family must be a CUDA-core one (0, 1, 2, 4)
    for rk in (-1, 3, 5):
        with pytest.raises(iaat.IaatError) as e:
            iaat.iaat_plan_create(_desc(), iaat.IAAT_F32, iaat.IAAT_PREC_3XBF16, route_k_below=8, route_kernel=rk)
        assert e.value.status == 1 and "route_kernel" in e.value.message


def test_kernel_option_range(L):
    """kernel 0..4; the warp-direct kernel (4) takes plans of the default
    precision only; all refused before any device work."""
    for k in (-1, 5):
        with pytest.raises(iaat.IaatError) as e:
            iaat.iaat_plan_create(_desc(), iaat.IAAT_F32, iaat.IAAT_PREC_DEFAULT, kernel=k)
        assert e.value.status == 1 and "kernel" in e.value.message
    with pytest.raises(iaat.IaatError) as e:
        iaat.iaat_plan_create(_desc(), iaat.IAAT_F32, iaat.IAAT_PREC_3XBF16, kernel=4)
    assert e.value.status == 1 and "warp-direct" in e.value.message


def test_pack_create_validates_before_the_device(L):
    with pytest.raises(iaat.IaatError) as e:
        iaat.iaat_pack_create(_desc(), iaat.IAAT_C32)
    assert e.value.status == 1
    with pytest.raises(iaat.IaatError) as e:
        iaat.iaat_pack_create(np.concatenate([_desc(), _desc(ldc=3)]), iaat.IAAT_F32)
    assert e.value.status == 1 and "instance 1" in e.value.message
    with pytest.raises(iaat.IaatError) as e:
        iaat.iaat_pack_create(_desc(M=80, N=80, K=81, lda=80, ldb=81, ldc=80), iaat.IAAT_F64)
    assert e.value.status == 2


def test_struct_layouts_match_the_header(tmp_path):
    """The Python mirrors of the header's structs (numpy descriptor dtypes,
    ctypes option and info structs) have the C compiler's sizes and field
    offsets."""
    import ctypes
    import subprocess
    fields = {
        "iaat_gemm_desc_t": (iaat.DESC_DTYPE, [n for n in iaat.DESC_DTYPE.names]),
        "iaat_cgemm_desc_t": (iaat.CDESC_DTYPE, [n for n in iaat.CDESC_DTYPE.names]),
    }
    src = ['#include <stdio.h>', '#include <stddef.h>', '#include "iaat.h"', 'int main(void) {']
    for st, (_, names) in fields.items():
        src.append(f'printf("{st} %zu\\n", sizeof({st}));')
        for n in names:
            src.append(f'printf("{st}.{n} %zu\\n", offsetof({st}, {n}));')
    for st, cls in (("iaat_plan_options_t", iaat.PlanOptions), ("iaat_plan_info_t", iaat.PlanInfo)):
        src.append(f'printf("{st} %zu\\n", sizeof({st}));')
        for n, _ in cls._fields_:
            src.append(f'printf("{st}.{n} %zu\\n", offsetof({st}, {n}));')
    src.append('return 0; }')
    c = tmp_path / "layout.c"
    c.write_text("\n".join(src))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c99", f"-I{os.path.join(ROOT, 'include')}", str(c), "-o", str(exe)])
    got = dict(line.split() for line in subprocess.check_output([str(exe)], text=True).splitlines())
    for st, (dt, names) in fields.items():
        assert int(got[st]) == dt.itemsize, st
        for n in names:
            assert int(got[f"{st}.{n}"]) == dt.fields[n][1], (st, n)
    for st, cls in (("iaat_plan_options_t", iaat.PlanOptions), ("iaat_plan_info_t", iaat.PlanInfo)):
        assert int(got[st]) == ctypes.sizeof(cls), st
        for n, _ in cls._fields_:
            assert int(got[f"{st}.{n}"]) == getattr(cls, n).offset, (st, n)


def test_single_complex_calls_reject_before_the_device(L):
    with pytest.raises(iaat.IaatError) as e:
        iaat.iaat_zgemm(0, 0, 81, 80, 80, 1.0, 0x1000, 81, 0x2000, 80, 0.0, 0x3000, 81)
    assert e.value.status == 2
    with pytest.raises(iaat.IaatError) as e:   # 8 bytes past 16: aligned for CGEMM, not ZGEMM
        iaat.iaat_zgemm(0, 0, 4, 4, 4, 1.0, 0x1008, 4, 0x2000, 4, 0.0, 0x3000, 4)
    assert e.value.status == 3
    with pytest.raises(iaat.IaatError) as e:
        iaat.iaat_cgemm(1, 0, 32, 32, 33, 1j, 0x1000, 33, 0x2000, 33, 0.0, 0x3000, 32)
    assert e.value.status == 2
    assert iaat.lib().iaat_cgemm(0, 0, 4, 4, 4, None, 0x1000, 4, 0x2000, 4, None, 0x3000, 4, None) == 1
    # quick returns touch nothing
    iaat.iaat_cgemm(0, 0, 0, 5, 5, 1.0, 0, 1, 0, 5, 0.0, 0, 1)
    iaat.iaat_zgemm(0, 0, 5, 5, 5, 0.0, 0, 5, 0, 5, 1.0, 0x3000, 5)
