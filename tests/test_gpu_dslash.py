"""GPU parity of the stencil operators (Dhop, Dhop^+, D, D^+, D^+D) against the
CPU oracle, through the C ABI, on the same seeded inputs.

Tolerances (relative L2 over each right-hand side): 1e-12 at FP64, 1e-5 at
FP32 storage, 5e-3 at FP16 storage.
"""

import itertools

import numpy as np
import pytest

import oracle
from gpu_helpers import (ALL_OPS, BC, OP_NAMES, STENCIL_OPS, TOL, build_library, make_case,
                         max_rel, run_gpu, run_oracle, valid_tiles)
from paper_2112_01852_gb300 import dw

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build_library()
    import torch
    assert torch.cuda.is_available()


def _lattice(dims, Ls, kind, prec, M5=1.8, b=1.5, c=0.5, bc=BC):
    from paper_2112_01852_gb300.lattice import Lattice
    return Lattice(dims, Ls, kind=kind, M5=M5, b=b, c=c, prec=prec, bc=bc)


# ---------------------------------------------------------------------------
# Shamir D_dw at FP64 on 4^4 x Ls=8, Haar links, seed 1, mf = 0.01


@pytest.mark.parametrize("op", ALL_OPS, ids=lambda o: OP_NAMES[o])
def test_shamir_4x4x4x4_ls8_f64(op):
    dims, Ls = (4, 4, 4, 4), 8
    U, psi = make_case(dims, Ls, 1, seed=1, links="haar")
    lat = _lattice(dims, Ls, dw.DW_SHAMIR, dw.DW_F64)
    lat.load_gauge(U)
    got = run_gpu(lat, op, psi, mf=[0.01])
    ref = run_oracle(op, psi, U, dims, Ls, 1.8, 1.0, 0.0, [0.01])
    assert max_rel(got, ref) <= TOL[dw.DW_F64]
    lat.close()


# ---------------------------------------------------------------------------
# Moebius (b=1.5, c=0.5) on 16^4 x Ls=16, exp(i 0.3 H) links, seed 2, FP64/FP32


@pytest.fixture(scope="module")
def case_16x4_ls16():
    dims, Ls = (16, 16, 16, 16), 16
    U, psi = make_case(dims, Ls, 1, seed=2)
    refs = {op: run_oracle(op, psi, U, dims, Ls, 1.8, 1.5, 0.5, [0.01]) for op in ALL_OPS}
    return dims, Ls, U, psi, refs


@pytest.mark.parametrize("prec", [dw.DW_F64, dw.DW_F32], ids=["f64", "f32"])
@pytest.mark.parametrize("op", ALL_OPS, ids=lambda o: OP_NAMES[o])
def test_mobius_16x4_ls16(case_16x4_ls16, prec, op):
    dims, Ls, U, psi, refs = case_16x4_ls16
    lat = _lattice(dims, Ls, dw.DW_MOBIUS, prec)
    lat.load_gauge(U)
    got = run_gpu(lat, op, psi, mf=[0.01])
    assert max_rel(got, refs[op]) <= TOL[prec]
    lat.close()


# ---------------------------------------------------------------------------
# Every tile on a ragged lattice (V4 = 210 is not a multiple of any tile),
# including Ls = 1 (the Wilson hop) and Ls = 12 (not a divisor of the warp).


@pytest.mark.parametrize("Ls", [1, 6, 12])
def test_all_tiles_ragged(Ls):
    dims = (3, 5, 2, 7)
    bc = (-1, 1, 1, -1)
    U, psi = make_case(dims, Ls, 2, seed=7)
    mfs = [0.02, 0.3]
    lat = _lattice(dims, Ls, dw.DW_MOBIUS, dw.DW_F64, M5=1.6, b=1.25, c=0.75, bc=bc)
    lat.load_gauge(U)
    refs = {op: run_oracle(op, psi, U, dims, Ls, 1.6, 1.25, 0.75, mfs, bc) for op in STENCIL_OPS}
    ran = set()
    for variant in range(8):
        for spt, tx in valid_tiles(Ls):
            for op in STENCIL_OPS:
                try:
                    lat.set_tile(op, spt, tx, variant, zblk=1 + (spt + tx // 32) % 2)
                except dw.DWError as e:  # variant not built at FP64, or CTA too large
                    assert e.code == dw.DW_ERR_ARG
                    continue
                ran.add((variant, op))
                got = run_gpu(lat, op, psi, mf=mfs)
                err = max_rel(got, refs[op])
                assert err <= TOL[dw.DW_F64], (OP_NAMES[op], spt, tx, variant, err)
    # FP64 builds the register variants 0 and 2; each ran for every operator
    assert {(v, op) for v in (0, 2) for op in STENCIL_OPS} <= ran
    lat.close()


@pytest.mark.parametrize("prec", [dw.DW_F64, dw.DW_F32, dw.DW_F16], ids=["f64", "f32", "f16"])
def test_slice_groups_equal_one_cta(prec):
    # splitting the slices of a tile over sgrp CTAs changes only which CTA
    # computes a site: the result is the same bit for bit
    dims, Ls = (8, 4, 6, 10), 12
    U, psi = make_case(dims, Ls, 2, seed=16)
    mfs = [0.01, 0.04]
    lat = _lattice(dims, Ls, dw.DW_MOBIUS, prec)
    lat.load_gauge(U)
    ran = 0
    # D^+: the slice groups of a tile form a thread-block cluster and exchange
    # their edge slices through distributed shared memory (sgrp <= 8)
    for op in (dw.DW_OP_DHOP, dw.DW_OP_DHOP_DAG, dw.DW_OP_D, dw.DW_OP_DDAG):
        for variant in range(8):
            for spt in (1, 2, 3):
                try:
                    lat.set_tile(op, spt, 32, variant)
                except dw.DWError:
                    continue
                ref = run_gpu(lat, op, psi, mf=mfs)
                for sgrp in (2, 3, 4, 6, 12):
                    if (Ls // spt) % sgrp or (op == dw.DW_OP_DDAG and sgrp > 8):
                        continue
                    lat.set_tile(op, spt, 32, variant, sgrp=sgrp)
                    got = run_gpu(lat, op, psi, mf=mfs)
                    assert np.array_equal(got, ref), (OP_NAMES[op], variant, spt, sgrp)
                    ran += 1
    assert ran > 0
    lat.close()


@pytest.mark.parametrize("prec", [dw.DW_F32, dw.DW_F16], ids=["f32", "f16"])
@pytest.mark.parametrize("dims", [(32, 4, 2, 6), (32, 2, 2, 4), (32, 1, 2, 4), (16, 4, 2, 4),
                                  (24, 4, 2, 4), (8, 8, 2, 4), (16, 2, 2, 4)],
                         ids=["Ly4", "Ly2", "Ly1", "Lx16", "Lx24", "Lx8", "one_block"])
def test_row_staged_variant(prec, dims):
    # variants 6 and 7 read the x and y neighbours from 32-site blocks of the
    # plane staged in shared memory (7 walking the plane's tiles with a ring of
    # blocks); they sum the same terms in the same order as variant 5: equal
    # bit for bit, and within tolerance of the oracle.  Ly = 2 and 1 at Lx = 32,
    # and a plane of one block: the halo blocks repeat blocks of the tile (and
    # the ring wraps within one step); Lx = 24: a block holds a row and a part.
    # D stages the s-neighbours of each CTA's slice range as well (wrapped in s
    # with the -m_f factor at sgrp 1, the first and the last slice group), and
    # takes its local term alpha psi + beta K psi from the staged own site.
    Ls = 4
    U, psi = make_case(dims, Ls, 2, seed=17)
    mfs = [0.03, 0.2]
    lat = _lattice(dims, Ls, dw.DW_MOBIUS, prec)
    lat.load_gauge(U)
    ran = 0
    for op in (dw.DW_OP_DHOP, dw.DW_OP_DHOP_DAG, dw.DW_OP_D):
        mf = mfs if op == dw.DW_OP_D else [0.0, 0.0]
        ref = run_oracle(op, psi, U, dims, Ls, 1.8, 1.5, 0.5, mf)
        for spt in (1, 2):
            lat.set_tile(op, spt, 32, 5)
            v5 = run_gpu(lat, op, psi, mf=mf)
            for var, tx, sgrp in itertools.product((6, 7), (32, 64, 128), (1, 2, 4)):
                try:
                    lat.set_tile(op, spt, tx, var, sgrp=sgrp)
                except dw.DWError as e:
                    assert e.code == dw.DW_ERR_ARG
                    continue
                got = run_gpu(lat, op, psi, mf=mf)
                assert np.array_equal(got, v5), (OP_NAMES[op], spt, tx, var, sgrp)
                assert max_rel(got, ref) <= TOL[prec]
                ran += 1
    dw.dw_device_status(lat.handle)
    assert ran >= 24
    for var in (6, 7):
        with pytest.raises(dw.DWError):  # D^+ combines all slices of a site after the hops
            lat.set_tile(dw.DW_OP_DDAG, 1, 32, var)
    lat.close()


@pytest.mark.parametrize("op, variant, sgrp",
                         [(dw.DW_OP_D, 6, 2), (dw.DW_OP_D, 7, 2), (dw.DW_OP_DDAG, 4, 2),
                          (dw.DW_OP_DDAG, 5, 4)],
                         ids=["D_v6", "D_v7", "Ddag_cluster2", "Ddag_cluster4"])
def test_forced_tiles_in_mixed_cg(op, variant, sgrp):
    # the mixed-precision CG with the D pass in a row-staged tile (its |D p|^2
    # CTA partials are summed over the steps of a ring CTA), or the D^+ pass
    # (which applies the residual update itself) in a tile whose slice groups
    # form a thread-block cluster: the solve reaches an oracle-recomputed
    # residual <= 1e-10 in the iterations of the default tiles
    dims, Ls, nrhs = (32, 4, 4, 4), 8, 2
    U, eta = make_case(dims, Ls, nrhs, seed=23)
    mfs = [0.1, 0.3]
    iters = {}
    for forced in (False, True):
        lat = _lattice(dims, Ls, dw.DW_MOBIUS, dw.DW_F64)
        lat.load_gauge(U)
        if forced:
            lat.set_tile(op, 2 if op == dw.DW_OP_D else 1, 64, variant, nrhs=nrhs,
                         prec=dw.DW_F32, sgrp=sgrp)
        b = lat.pack(eta)
        x = lat.empty(nrhs)
        x.zero_()
        rc, stats = lat.cg(x, b, mfs, nrhs, tol=1e-10, maxit=2000, mode=dw.DW_F32)
        assert rc == dw.DW_OK and all(st.converged for st in stats)
        xs = lat.unpack(x, nrhs)
        lat.close()
        Ax = oracle.dwdagdw(xs, U, dims, Ls, 1.8, 1.5, 0.5, mfs, BC)
        for r in range(nrhs):
            rel = np.linalg.norm((eta[r] - Ax[r]).ravel()) / np.linalg.norm(eta[r].ravel())
            assert rel <= 1e-10, (forced, r, rel)
        iters[forced] = [st.iters for st in stats]
    assert all(abs(a - b) <= 2 for a, b in zip(iters[True], iters[False])), iters


@pytest.mark.parametrize("dims", [(48, 2, 2, 4), (12, 4, 2, 4)], ids=["Lx48", "plane48"])
def test_row_staged_variant_limits(dims):
    # Lx > 32 (a y neighbour two blocks away) or a plane that is not a whole
    # number of 32-site blocks: the row-staged variants refuse the tile
    Ls = 4
    U, _ = make_case(dims, Ls, 1, seed=18)
    lat = _lattice(dims, Ls, dw.DW_MOBIUS, dw.DW_F32)
    lat.load_gauge(U)
    for var in (6, 7):
        with pytest.raises(dw.DWError) as e:
            lat.set_tile(dw.DW_OP_DHOP, 1, 32, var)
        assert e.value.code == dw.DW_ERR_ARG
    lat.close()


@pytest.mark.parametrize("op", [dw.DW_OP_DHOP, dw.DW_OP_DHOP_DAG, dw.DW_OP_D],
                         ids=["Dhop", "Dhop_dag", "D"])
def test_bounded_wait_timeout_is_reported(op):
    # With the first bounded wait of each step limited to zero polls, every
    # row-staged launch gives up that wait: the kernel records the timeout in
    # the lattice's status word (DW_ERR_TIMEOUT from dw_device_status, once),
    # then its second bounded wait lets the copies in flight land, so the
    # result is still right.  With the built-in bound restored the status stays
    # clear.
    dims, Ls = (32, 4, 2, 4), 4
    U, psi = make_case(dims, Ls, 1, seed=19)
    mf = [0.05] if op == dw.DW_OP_D else [0.0]
    ref = run_oracle(op, psi, U, dims, Ls, 1.8, 1.5, 0.5, mf)
    lat = _lattice(dims, Ls, dw.DW_MOBIUS, dw.DW_F32)
    lat.load_gauge(U)
    with pytest.raises(dw.DWError) as e:
        dw.dw_set_wait_polls(lat.handle, -2)
    assert e.value.code == dw.DW_ERR_ARG
    for var in (6, 7):
        lat.set_tile(op, 1, 32, var)
        dw.dw_device_status(lat.handle)
        dw.dw_set_wait_polls(lat.handle, 0)
        got = run_gpu(lat, op, psi, mf=mf)
        with pytest.raises(dw.DWError) as e:
            dw.dw_device_status(lat.handle)
        assert e.value.code == dw.DW_ERR_TIMEOUT, var
        dw.dw_device_status(lat.handle)  # read and cleared: no second report
        assert max_rel(got, ref) <= TOL[dw.DW_F32], var
        dw.dw_set_wait_polls(lat.handle, -1)
        got = run_gpu(lat, op, psi, mf=mf)
        dw.dw_device_status(lat.handle)
        assert max_rel(got, ref) <= TOL[dw.DW_F32], var
    lat.close()


def test_two_site_lattice_sums_coinciding_neighbours():
    # On a 2^4 lattice x+mu and x-mu are the same site: both hops must add.
    dims, Ls = (2, 2, 2, 2), 4
    U, psi = make_case(dims, Ls, 1, seed=8, links="haar")
    lat = _lattice(dims, Ls, dw.DW_MOBIUS, dw.DW_F64)
    lat.load_gauge(U)
    for op in ALL_OPS:
        got = run_gpu(lat, op, psi, mf=[0.05])
        ref = run_oracle(op, psi, U, dims, Ls, 1.8, 1.5, 0.5, [0.05])
        assert max_rel(got, ref) <= TOL[dw.DW_F64], OP_NAMES[op]
    lat.close()


@pytest.mark.parametrize("prec", [dw.DW_F32, dw.DW_F16], ids=["f32", "f16"])
def test_both_variants_low_precision(prec):
    dims, Ls = (8, 4, 6, 10), 12
    U, psi = make_case(dims, Ls, 2, seed=15)
    mfs = [0.01, 0.04]
    lat = _lattice(dims, Ls, dw.DW_MOBIUS, prec)
    lat.load_gauge(U)
    refs = {op: run_oracle(op, psi, U, dims, Ls, 1.8, 1.5, 0.5, mfs) for op in STENCIL_OPS}
    ran = set()
    for variant in range(8):
        for spt in (1, 2, 3, 4):
            for op in STENCIL_OPS:
                try:
                    lat.set_tile(op, spt, 32, variant)
                except dw.DWError:
                    continue
                ran.add((variant, op))
                got = run_gpu(lat, op, psi, mf=mfs)
                assert max_rel(got, refs[op]) <= TOL[prec], (OP_NAMES[op], spt, variant)
    built = tuple(range(6))  # variants 6, 7 need Lx = 32: their own test below
    assert {(v, op) for v in built for op in STENCIL_OPS} <= ran
    lat.close()


# ---------------------------------------------------------------------------
# FP16 storage with FP32 arithmetic


@pytest.mark.parametrize("op", ALL_OPS, ids=lambda o: OP_NAMES[o])
def test_f16_storage(op):
    dims, Ls = (8, 8, 8, 8), 8
    U, psi = make_case(dims, Ls, 1, seed=9)
    lat = _lattice(dims, Ls, dw.DW_MOBIUS, dw.DW_F16)
    lat.load_gauge(U)
    got = run_gpu(lat, op, psi, mf=[0.01])
    ref = run_oracle(op, psi, U, dims, Ls, 1.8, 1.5, 0.5, [0.01])
    assert max_rel(got, ref) <= TOL[dw.DW_F16]
    lat.close()


# ---------------------------------------------------------------------------
# Several right-hand sides with uneven mass counts (5/4/2/1 over 4 masses)


def test_multi_rhs_uneven_masses_f32():
    dims, Ls = (4, 4, 4, 8), 12
    mfs = [0.005] * 5 + [0.01] * 4 + [0.02] * 2 + [0.05]
    U, psi = make_case(dims, Ls, len(mfs), seed=4)
    lat = _lattice(dims, Ls, dw.DW_MOBIUS, dw.DW_F32)
    lat.load_gauge(U)
    for op in ALL_OPS:
        got = run_gpu(lat, op, psi, mf=mfs)
        ref = run_oracle(op, psi, U, dims, Ls, 1.8, 1.5, 0.5, mfs)
        assert max_rel(got, ref) <= TOL[dw.DW_F32], OP_NAMES[op]
    lat.close()


def test_more_rhs_than_one_launch():
    # 70 RHS are split into launches of at most 64
    dims, Ls = (2, 2, 2, 4), 2
    nrhs = 70
    mfs = list(np.linspace(0.01, 0.7, nrhs))
    U, psi = make_case(dims, Ls, nrhs, seed=10)
    lat = _lattice(dims, Ls, dw.DW_MOBIUS, dw.DW_F64)
    lat.load_gauge(U)
    for op in (dw.DW_OP_DHOP, dw.DW_OP_D, dw.DW_OP_DDAG):
        got = run_gpu(lat, op, psi, mf=mfs)
        ref = run_oracle(op, psi, U, dims, Ls, 1.8, 1.5, 0.5, mfs)
        assert max_rel(got, ref) <= TOL[dw.DW_F64], OP_NAMES[op]
    lat.close()


# ---------------------------------------------------------------------------
# Layout round trips, host-buffer path, tuner, argument errors


def test_pack_unpack_roundtrip():
    dims, Ls = (4, 2, 6, 2), 3
    _, psi = make_case(dims, Ls, 2, seed=11)
    lat = _lattice(dims, Ls, dw.DW_MOBIUS, dw.DW_F64)
    for prec in (dw.DW_F64, dw.DW_F32, dw.DW_F16):
        back = lat.unpack(lat.pack(psi, prec), 2, prec)
        if prec == dw.DW_F64:
            assert np.array_equal(back, psi)
        elif prec == dw.DW_F32:
            assert np.array_equal(back.real, psi.real.astype(np.float32).astype(np.float64))
            assert np.array_equal(back.imag, psi.imag.astype(np.float32).astype(np.float64))
        else:
            assert np.array_equal(back.real, psi.real.astype(np.float16).astype(np.float64))
            assert np.array_equal(back.imag, psi.imag.astype(np.float16).astype(np.float64))
    lat.close()


def test_apply_host_matches_device():
    import torch
    dims, Ls = (8, 4, 4, 8), 8
    U, psi = make_case(dims, Ls, 2, seed=12)
    lat = _lattice(dims, Ls, dw.DW_MOBIUS, dw.DW_F32)
    lat.load_gauge(U)
    x = lat.pack(psi)
    for op in ALL_OPS:
        dev = run_gpu(lat, op, psi, mf=[0.01, 0.02])
        hin = x.cpu().pin_memory()
        hout = torch.empty_like(hin).pin_memory()
        lat.apply_host(op, hout, hin, mf=None if op < dw.DW_OP_D else [0.01, 0.02], nrhs=2)
        host = lat.unpack(hout.cuda(), 2)
        assert np.array_equal(host, dev), OP_NAMES[op]
    lat.close()


@pytest.mark.parametrize("dims", [(16, 16, 8, 16), (32, 16, 16, 16), (16, 16, 16, 6),
                                  (32, 16, 16, 40)],
                         ids=["4slabs", "16slabs_T1", "3slabs", "40slabs_T1"])
def test_apply_host_slab_pipeline_matches_device(dims):
    # Lx Ly Lz a multiple of 32: the host apply moves the field in t slabs
    # (4, 16 of one time slice, 3, 40 of one slice) and must equal the device
    # apply bit for bit
    import torch
    Ls = 4
    U, psi = make_case(dims, Ls, 2, seed=14)
    lat = _lattice(dims, Ls, dw.DW_MOBIUS, dw.DW_F32)
    lat.load_gauge(U)
    x = lat.pack(psi)
    hin = x.cpu().pin_memory()
    hout = torch.empty_like(hin).pin_memory()
    for op in ALL_OPS:
        dev = run_gpu(lat, op, psi, mf=[0.01, 0.02])
        hout.zero_()
        lat.apply_host(op, hout, hin, mf=None if op < dw.DW_OP_D else [0.01, 0.02], nrhs=2)
        host = lat.unpack(hout.cuda(), 2)
        assert np.array_equal(host, dev), OP_NAMES[op]
    lat.close()


def test_tune_picks_valid_tile_and_stays_exact():
    dims, Ls = (8, 8, 8, 8), 12
    U, psi = make_case(dims, Ls, 1, seed=13)
    lat = _lattice(dims, Ls, dw.DW_MOBIUS, dw.DW_F32)
    lat.load_gauge(U)
    for op in STENCIL_OPS:
        spt, tx, variant, zblk, sgrp = lat.tune(op, 1)
        assert dims[2] % zblk == 0
        assert Ls % spt == 0 and tx % 32 == 0 and tx * (Ls // spt) <= 1024
        assert (Ls // spt) % sgrp == 0 and (sgrp <= 8 or op != dw.DW_OP_DDAG)
        assert variant in range(8)
        got = run_gpu(lat, op, psi, mf=[0.01])
        ref = run_oracle(op, psi, U, dims, Ls, 1.8, 1.5, 0.5, [0.01])
        assert max_rel(got, ref) <= TOL[dw.DW_F32], OP_NAMES[op]
    lat.close()


def test_argument_errors():
    import torch
    dims, Ls = (4, 4, 4, 4), 4
    with pytest.raises(dw.DWError) as e:
        dw.dw_create_lattice((4, 0, 4, 4), 4, dw.DW_MOBIUS, 1.8, 1.5, 0.5, dw.DW_F32)
    assert e.value.code == dw.DW_ERR_ARG
    with pytest.raises(dw.DWError) as e:
        dw.dw_create_lattice(dims, 0, dw.DW_MOBIUS, 1.8, 1.5, 0.5, dw.DW_F32)
    assert e.value.code == dw.DW_ERR_ARG
    with pytest.raises(dw.DWError) as e:
        dw.dw_create_lattice(dims, 4, dw.DW_MOBIUS, 1.8, 1.5, 0.5, 7)
    assert e.value.code == dw.DW_ERR_ARG
    with pytest.raises(dw.DWError) as e:
        dw.dw_create_lattice(dims, 4, dw.DW_MOBIUS, 1.8, 1.5, 0.5, dw.DW_F32, bc=(1, 1, 2, -1))
    assert e.value.code == dw.DW_ERR_ARG
    lat = _lattice(dims, Ls, dw.DW_MOBIUS, dw.DW_F32)
    x = lat.empty(1)
    y = lat.empty(1)
    with pytest.raises(dw.DWError) as e:  # gauge not loaded yet
        lat.dhop(y, x)
    assert e.value.code == dw.DW_ERR_STATE
    U, _ = make_case(dims, Ls, 1, seed=14)
    lat.load_gauge(U)
    with pytest.raises(dw.DWError) as e:  # aliasing
        lat.dhop(x, x)
    assert e.value.code == dw.DW_ERR_ARG
    with pytest.raises(dw.DWError) as e:  # misaligned
        dw.dw_apply_Dhop(lat.handle, y.data_ptr() + 4, x.data_ptr(), 1)
    assert e.value.code == dw.DW_ERR_ARG
    with pytest.raises(dw.DWError) as e:  # null mass array
        dw.dw_apply_D(lat.handle, y.data_ptr(), x.data_ptr(), None, 1)
    assert e.value.code == dw.DW_ERR_ARG
    with pytest.raises(dw.DWError) as e:
        lat.set_tile(dw.DW_OP_DHOP, 3, 32)  # 3 does not divide Ls = 4
    assert e.value.code == dw.DW_ERR_ARG
    with pytest.raises(dw.DWError) as e:
        lat.set_tile(dw.DW_OP_DHOP, 1, 48)  # not a multiple of 32
    assert e.value.code == dw.DW_ERR_ARG
    with pytest.raises(dw.DWError) as e:
        lat.set_tile(dw.DW_OP_DHOP, 1, 32, variant=9)
    assert e.value.code == dw.DW_ERR_ARG
    with pytest.raises(dw.DWError) as e:
        lat.set_tile(dw.DW_OP_DHOP, 1, 32, zblk=3)  # 3 does not divide Lz = 4
    assert e.value.code == dw.DW_ERR_ARG
    with pytest.raises(dw.DWError) as e:
        lat.set_tile(dw.DW_OP_DHOP, 1, 32, sgrp=3)  # 3 does not divide Ls / spt = 4
    assert e.value.code == dw.DW_ERR_ARG
    assert "multiple" in dw.dw_last_error() or "invalid" in dw.dw_last_error()
    torch.cuda.synchronize()
    lat.close()
    # D^+ spreads a tile's slice groups over a thread-block cluster of sgrp CTAs:
    # at most the portable cluster size, 8
    lat16 = _lattice(dims, 16, dw.DW_MOBIUS, dw.DW_F32)
    lat16.set_tile(dw.DW_OP_DDAG, 1, 32, sgrp=8)
    with pytest.raises(dw.DWError) as e:
        lat16.set_tile(dw.DW_OP_DDAG, 1, 32, sgrp=16)
    assert e.value.code == dw.DW_ERR_ARG
    lat16.close()
