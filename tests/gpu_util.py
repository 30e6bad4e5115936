"""Helpers of the GPU parity tests: move a batch to the device, run it through
the C ABI, gather results and compare them with the FP64 oracle."""
from __future__ import annotations

import numpy as np

import oracle
from paper_2208_09822_gb300 import iaat
from paper_2208_09822_gb300 import workloads as W


def gather_index(batch, which, idx=None):
    """Pool indices of the elements of every selected stored matrix, each
    instance's block column-major and tight, concatenated; plus the
    per-instance element counts."""
    rows, cols, ld, off = batch.storage(which)
    if idx is None:
        idx = np.arange(batch.count)
    rows, cols, ld, off = rows[idx], cols[idx], ld[idx], off[idx]
    cnt = rows * cols
    tot = int(cnt.sum())
    inst = np.repeat(np.arange(len(idx)), cnt)
    first = np.zeros(len(idx), np.int64)
    if len(idx) > 1:
        first[1:] = np.cumsum(cnt)[:-1]
    loc = np.arange(tot, dtype=np.int64) - first[inst]
    rr = np.maximum(rows[inst], 1)
    return off[inst] + (loc // rr) * ld[inst] + loc % rr, cnt


DTYPES = {np.float32: iaat.IAAT_F32, np.float64: iaat.IAAT_F64,
          np.complex64: iaat.IAAT_C32, np.complex128: iaat.IAAT_C64}


def to_device(batch):
    import torch
    dev = torch.device("cuda:0")
    tA = torch.from_numpy(batch.A).to(dev)
    tB = torch.from_numpy(batch.B).to(dev)
    tC = torch.from_numpy(batch.C).to(dev)
    make = iaat.cdescs_for_pools if batch.is_complex else iaat.descs_for_pools
    descs = make(batch, tA.data_ptr(), tB.data_ptr(), tC.data_ptr())
    return tA, tB, tC, descs


def plan_for(batch, descs, precision=iaat.IAAT_PREC_DEFAULT, **plan_kw):
    """iaat_plan_create, or iaat_plan_create_complex for a complex batch."""
    dtype = DTYPES[np.dtype(batch.dtype).type]
    if batch.is_complex:
        return iaat.iaat_plan_create_complex(descs, dtype, **plan_kw)
    return iaat.iaat_plan_create(descs, dtype, precision, **plan_kw)


def run_grouped(batch, precision=iaat.IAAT_PREC_DEFAULT, **plan_kw):
    """Plan + one grouped launch + check; returns the C pool (numpy) and the
    plan info."""
    import torch
    tA, tB, tC, descs = to_device(batch)
    plan = plan_for(batch, descs, precision, **plan_kw)
    s = torch.cuda.current_stream()
    iaat.iaat_gemm_grouped(plan, s)
    iaat.iaat_plan_check(plan, s)
    info = iaat.iaat_plan_info(plan)
    out = tC.cpu().numpy()
    plan.destroy()
    return out, info


def compare(batch, Cpool, idx=None, nthreads=0):
    """Errors of the GPU result against the oracle on instances idx."""
    if idx is None:
        idx = np.arange(batch.count)
    run = oracle.cgemm_batch if batch.is_complex else oracle.gemm_batch
    ref, _ = run(batch, idx, nthreads=nthreads)
    return errors(batch, Cpool, ref, idx)


def errors(batch, Cpool, ref, idx=None):
    """Errors of a result pool against reference values ``ref`` (the
    oracle's tight MxN blocks of instances idx, concatenated).

    Returns dict: eps_batch = ||dC||_F / ||C_ref||_F over the selection, and
    the per-instance guarded error
    eps_i = ||dC_i||_F / (|alpha| ||opA_i||_F ||opB_i||_F + |beta| ||C0_i||_F)
    (max, median, rms), plus 'exact' (all elements equal).  Complex batches
    take complex differences and moduli."""
    if idx is None:
        idx = np.arange(batch.count)
    cast = np.complex128 if np.iscomplexobj(Cpool) else np.float64
    gi, cnt = gather_index(batch, "C", idx)
    got = Cpool[gi].astype(cast)
    d = got - ref
    nref = np.linalg.norm(ref)
    ndiff = np.linalg.norm(d)
    eps_batch = ndiff / nref if nref > 0 else (0.0 if ndiff == 0 else np.inf)
    # guarded per-instance error
    starts = np.zeros(len(idx), np.int64)
    if len(idx) > 1:
        starts[1:] = np.cumsum(cnt)[:-1]

    def seg_norm(v, counts):
        s = np.zeros(len(counts))
        nz = counts > 0
        st = np.zeros(len(counts), np.int64)
        if len(counts) > 1:
            st[1:] = np.cumsum(counts)[:-1]
        if nz.any():
            s[nz] = np.add.reduceat(np.abs(v) ** 2, st[nz])[: nz.sum()] if len(v) else 0
        return np.sqrt(s)

    dn = seg_norm(d, cnt)
    ia, ca = gather_index(batch, "A", idx)
    ib, cb = gather_index(batch, "B", idx)
    nA = seg_norm(batch.A[ia].astype(cast), ca)
    nB = seg_norm(batch.B[ib].astype(cast), cb)
    nC = seg_norm(batch.C[gi].astype(cast), cnt)
    al = np.abs(batch.alpha[idx])
    be = np.abs(batch.beta[idx])
    den = al * nA * nB + be * nC
    with np.errstate(divide="ignore", invalid="ignore"):
        epsi = np.where(den > 0, dn / np.where(den > 0, den, 1), np.where(dn > 0, np.inf, 0.0))
    return {
        "eps_batch": float(eps_batch),
        "eps_inst_max": float(epsi.max()) if len(epsi) else 0.0,
        "eps_inst_median": float(np.median(epsi)) if len(epsi) else 0.0,
        "eps_inst_rms": float(np.sqrt(np.mean(epsi ** 2))) if len(epsi) else 0.0,
        "exact": bool(np.array_equal(got, ref)),
        "nan": bool(np.isnan(got).any()),
    }


def padding_untouched(batch, Cpool):
    """Every C pool element outside the batch's M x N parts (ld padding, gaps
    between matrices, instances not in the batch) is bit-identical to the
    input pool."""
    gi, _ = gather_index(batch, "C")
    mask = np.ones(len(Cpool), bool)
    mask[gi] = False
    a = Cpool[mask].view(np.uint8)
    b = batch.C[mask].view(np.uint8)
    return bool(np.array_equal(a, b))
