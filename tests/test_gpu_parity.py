"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Bar (Section 2.2 makes every exact [[U,V,W]] reproduce A B in exact
arithmetic):
  * integer inputs in {-4..4}: bit-exact with the oracle's classical product
    for every algorithm, depth, scheme and tile (all intermediates are
    dyadic and far below 2^53);
  * uniform[-1,1] inputs: e_F = ||C - C_oracle||_F / ||C_oracle||_F <= 1e-11
    at <= 3 levels, and the classical kernel within 2 gamma_k |A||B|;
  * full-size products: sampled entries against the oracle's per-entry dot
    products.
"""
import glob
import os

import numpy as np
import pytest

import oracle
from oracle import norms, ozaki
import paper_1409_2908_gb300 as fmm
from paper_1409_2908_gb300 import synth
from tests.gpu_util import classical_bound, to_dev

pytestmark = pytest.mark.gpu

TOL_F = 1e-11
ALGS = sorted(os.path.basename(p)[:-4] for p in glob.glob(os.path.join(fmm.ALGORITHM_DIR, "*.fmm")))
SCHEMES = {"fused": fmm.FLAG_FUSED_ST | fmm.FLAG_FUSED_W, "write_once": 0,
           "fused_st_only": fmm.FLAG_FUSED_ST, "fused_w_only": fmm.FLAG_FUSED_W,
           "levelwise": fmm.FLAG_LEVELWISE,
           "levelwise_fused_w": fmm.FLAG_LEVELWISE | fmm.FLAG_FUSED_W,
           "levelwise_fused_st": fmm.FLAG_LEVELWISE | fmm.FLAG_FUSED_ST}


def run(plan, A, B):
    import torch
    C = fmm.gemm(plan, to_dev(A), to_dev(B))
    torch.cuda.synchronize()
    return C.cpu().numpy()


def base_case(name):
    from oracle import tensor
    M, K, N, R, *_ = tensor.load_fmm(fmm.algorithm_path(name))
    return M, K, N, R


@pytest.mark.parametrize("m,k,n", [(1, 1, 1), (7, 13, 5), (128, 128, 128), (130, 257, 66), (300, 17, 513),
                                   (40, 300, 7), (2, 5000, 300), (300, 3, 400), (33, 65, 31), (1000, 900, 32),
                                   (32, 700, 1000)])
def test_classical_integer_exact(m, k, n):
    # includes the thin shapes of the peeling fringes (<= 32 rows, columns or k)
    A, B = synth.operands(m, k, n, 1409, kind="integer")
    import torch
    C = fmm.classical_gemm(to_dev(A), to_dev(B))
    torch.cuda.synchronize()
    assert np.array_equal(C.cpu().numpy(), oracle.gemm(A, B))


@pytest.mark.parametrize("m,k,n", [(64, 64, 64), (129, 700, 95), (512, 512, 512)])
def test_classical_random_bound(m, k, n):
    A, B = synth.operands(m, k, n, 1410)
    import torch
    C = fmm.classical_gemm(to_dev(A), to_dev(B))
    torch.cuda.synchronize()
    assert np.all(np.abs(C.cpu().numpy() - oracle.gemm(A, B)) <= classical_bound(A, B))


@pytest.mark.parametrize("tile", [t for t in fmm.TILES if t != "auto"])
def test_every_tile_integer_exact(tile):
    p = fmm.Plan("strassen_222_7", levels=1, tile=tile)
    A, B = synth.operands(2 * 97 + 1, 2 * 61, 2 * 83 + 1, 5, kind="integer")
    assert np.array_equal(run(p, A, B), oracle.gemm(A, B))


def test_config_strassen_512():
    # Strassen <2,2,2;7>, one level, 512^3: integer copy bit-exact, uniform within tolerance
    p = fmm.Plan("strassen_222_7", levels=1)
    A, B = synth.operands(512, 512, 512, 1409, kind="integer")
    assert np.array_equal(run(p, A, B), oracle.gemm(A, B))
    A, B = synth.operands(512, 512, 512, 1409)
    C = oracle.gemm(A, B)
    Cg = run(p, A, B)
    assert norms.rel_frobenius(Cg, C) <= TOL_F
    assert np.all(np.abs(Cg - C) <= 8 * classical_bound(A, B) + 1e-14)


@pytest.mark.parametrize("name", ALGS)
@pytest.mark.parametrize("levels", [1, 2, 3])
@pytest.mark.parametrize("scheme", list(SCHEMES))
def test_fast_integer_exact_ragged(name, levels, scheme):
    M, K, N, R = base_case(name)
    if R ** levels > 20000:
        pytest.skip("too many leaves for this size")
    p = fmm.Plan(name, levels=levels, flags=SCHEMES[scheme])
    # several leaf tiles plus a ragged fringe in every dimension
    m = M ** levels * max(3, 160 // M ** levels) + 1
    k = K ** levels * max(3, 96 // K ** levels) + 3
    n = N ** levels * max(3, 140 // N ** levels) + 2
    A, B = synth.operands(m, k, n, 1409 + levels, kind="integer")
    assert np.array_equal(run(p, A, B), oracle.gemm(A, B))


@pytest.mark.parametrize("name", ALGS)
@pytest.mark.parametrize("levels", [1, 2, 3])
@pytest.mark.parametrize("scheme", ["fused", "levelwise", "levelwise_fused_w"])
def test_fast_uniform_tolerance(name, levels, scheme):
    M, K, N, R = base_case(name)
    if R ** levels > 20000:
        pytest.skip("too many leaves for this size")
    p = fmm.Plan(name, levels=levels, flags=SCHEMES[scheme])
    m, k, n = M ** levels * 40 + 5, K ** levels * 40 + 1, N ** levels * 40 + 7
    A, B = synth.operands(m, k, n, 2000 + levels)
    C = oracle.gemm(A, B)
    e = norms.rel_frobenius(run(p, A, B), C)
    assert e <= TOL_F, e


@pytest.mark.parametrize("flags", [fmm.FLAG_FUSED_ST, fmm.FLAG_LEVELWISE, 0])
def test_stored_product_schemes_are_deterministic(flags):
    p = fmm.Plan("strassen_222_7", levels=2, flags=flags)
    A, B = synth.operands(600, 520, 610, 9)
    c1 = run(p, A, B)
    c2 = run(p, A, B)
    assert np.array_equal(c1, c2)
    assert norms.rel_frobenius(c1, oracle.gemm(A, B)) <= TOL_F


def test_levels0_plan_is_classical():
    p = fmm.Plan("strassen_222_7", levels=0)
    A, B = synth.operands(77, 66, 55, 3, kind="integer")
    assert np.array_equal(run(p, A, B), oracle.gemm(A, B))


@pytest.mark.parametrize("m,k,n", [(1, 1, 1), (3, 3, 3), (1, 512, 1), (512, 1, 512), (9, 600, 7), (600, 7, 9)])
def test_degenerate_shapes(m, k, n):
    # problems smaller than M^L in some dimension take the classical path or
    # a fringe-only split
    p = fmm.Plan("strassen_222_7", levels=3)
    A, B = synth.operands(m, k, n, 11, kind="integer")
    assert np.array_equal(run(p, A, B), oracle.gemm(A, B))


def test_leading_dimensions_and_views():
    import torch
    p = fmm.Plan("strassen_222_7", levels=2)
    big = synth.matrix(700, 900, 4, kind="integer")
    Ad = to_dev(big)[3:303, 5:405]       # 300 x 400, lda 900
    Bd = to_dev(big)[100:500, 10:610]    # 400 x 600, ldb 900
    Cd = torch.zeros((350, 700), dtype=torch.float64, device="cuda")
    fmm.gemm(p, Ad, Bd, C=Cd[10:310, 50:650])
    torch.cuda.synchronize()
    A = big[3:303, 5:405]
    B = big[100:500, 10:610]
    out = Cd.cpu().numpy()
    assert np.array_equal(out[10:310, 50:650], oracle.gemm(np.ascontiguousarray(A), np.ascontiguousarray(B)))
    # nothing outside the C view was touched
    mask = np.ones_like(out, bool)
    mask[10:310, 50:650] = False
    assert np.all(out[mask] == 0)


def test_side_stream_and_launch_count():
    import torch
    p = fmm.Plan("strassen_222_7", levels=1)
    A, B = synth.operands(259, 257, 261, 12, kind="integer")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        Ad, Bd = to_dev(A), to_dev(B)
        C = fmm.gemm(p, Ad, Bd, stream=s)
    s.synchronize()
    assert np.array_equal(C.cpu().numpy(), oracle.gemm(A, B))
    # k-fringe init, core, row fringe, column fringe
    assert fmm.last_launch_count() == 4


def test_host_entry_point():
    import torch
    p = fmm.Plan("strassen_222_7", levels=2)
    A, B = synth.operands(333, 222, 444, 13, kind="integer")
    At = torch.from_numpy(A).pin_memory()
    Bt = torch.from_numpy(B).pin_memory()
    Ct = torch.empty((333, 444), dtype=torch.float64).pin_memory()
    ws = torch.empty(fmm.host_workspace_size(p, 333, 222, 444), dtype=torch.uint8, device="cuda")
    fmm.gemm_host(p, At, Bt, Ct, ws)
    assert np.array_equal(Ct.numpy(), oracle.gemm(A, B))
    fmm.gemm_host(None, At, Bt, Ct, ws)
    assert np.array_equal(Ct.numpy(), oracle.gemm(A, B))


@pytest.mark.parametrize("name,levels,m,k,n", [
    ("strassen_222_7", 1, 4096, 256, 4096),   # C out in 4 row bands of 2 block rows
    ("fmm_323_15", 1, 4080, 256, 4080),       # 3 uneven bands of 3 block rows
    ("strassen_222_7", 0, 3000, 300, 2900),   # classical emulation: 2 bands of one block row
    ("strassen_222_7", 1, 4097, 257, 4095),   # fringe: all of A awaited up front, C copied out whole
    ("strassen_222_7", 2, 1000, 512, 900),    # small: one band
    ("strassen_222_7", 1, 4096, 4096, 1024),  # A in 2 bands of 2 block rows behind B
    ("fmm_323_15", 1, 6003, 2800, 1200),      # A in 2 uneven bands of 3 block rows
    ("strassen_222_7", 0, 8190, 4100, 300),   # A in 4 bands, classical emulation
])
def test_host_entry_point_emulated(name, levels, m, k, n):
    # the overlapped host path (B copied while the A side runs, C copied out
    # in bands) gives the device entry point's result bit for bit, exact on
    # integer inputs, with packed and with strided host buffers
    import torch
    p = fmm.Plan(name, levels=levels, precision="ozaki_bf16")
    A, B = synth.operands(m, k, n, 14, kind="integer")
    Cd = fmm.gemm(p, to_dev(A), to_dev(B))
    torch.cuda.synchronize()
    Cd = Cd.cpu().numpy()
    ws = torch.empty(fmm.host_workspace_size(p, m, k, n), dtype=torch.uint8, device="cuda")
    rng = np.random.default_rng(5)
    rows, cols = rng.integers(0, m, 200), rng.integers(0, n, 200)
    exact, _ = oracle.gemm_entries(A, B, rows, cols)
    # pipeline depths: from the sizes, none, ragged bands, products in as
    # many bands as C
    try:
        for pad, (bands, gemm_bands) in [(0, (0, 0)), (3, (0, 0)), (0, (1, 1)), (3, (5, 3)), (0, (8, 8))]:
            fmm.set_host_pipeline(bands, gemm_bands)
            Ah = torch.zeros((m, k + pad), dtype=torch.float64).pin_memory()
            Bh = torch.zeros((k, n + pad), dtype=torch.float64).pin_memory()
            Ch = torch.full((m, n + pad), 7.0, dtype=torch.float64).pin_memory()
            Ah[:, :k] = torch.from_numpy(A)
            Bh[:, :n] = torch.from_numpy(B)
            for _ in range(2):
                fmm.gemm_host(p, Ah[:, :k], Bh[:, :n], Ch[:, :n], ws)
                C = Ch[:, :n].numpy()
                assert np.array_equal(C, Cd)
                assert np.array_equal(C[rows, cols], exact)
                assert bool((Ch[:, n:] == 7.0).all())
                Ch[:, :n] = 0.0
    finally:
        fmm.set_host_pipeline(0, 0)
    fmm.check_device_error()


@pytest.mark.parametrize("name,levels", [("strassen_222_7", 3), ("strassen_222_7", 1)])
def test_full_size_8192_sampled(name, levels):
    # the square 8192^3 workload in the benchmark's launch configuration,
    # checked on sampled entries against the oracle's per-entry dot products
    import torch
    m = k = n = 8192
    A, B = synth.operands(m, k, n, 1410)
    p = fmm.Plan(name, levels=levels)
    C = fmm.gemm(p, to_dev(A), to_dev(B))
    torch.cuda.synchronize()
    rows, cols = synth.sample_indices(m, n, 512, 77)
    e64, eld = oracle.gemm_entries(A, B, rows, cols)
    got = C[torch.from_numpy(rows).cuda(), torch.from_numpy(cols).cuda()].cpu().numpy()
    err = np.abs(got - eld)
    # normwise: the sampled error relative to the sampled values' magnitude
    assert np.linalg.norm(err) / np.linalg.norm(eld) <= TOL_F
    Ci = fmm.gemm(p, to_dev(np.rint(4 * A)), to_dev(np.rint(4 * B)))
    torch.cuda.synchronize()
    gi = Ci[torch.from_numpy(rows).cuda(), torch.from_numpy(cols).cuda()].cpu().numpy()
    ei64, _ = oracle.gemm_entries(np.rint(4 * A), np.rint(4 * B), rows, cols)
    assert np.array_equal(gi, ei64)


@pytest.mark.parametrize("name,levels,shape", [("strassen_222_7", 2, (256, 512, 384)),
                                                ("strassen_222_7", 1, (257, 131, 199)),
                                                ("fmm_323_15", 1, (300, 200, 303))])
def test_batched_one_grouped_launch(name, levels, shape):
    import torch
    m, k, n = shape
    p = fmm.Plan(name, levels=levels)
    ins = [synth.operands(m, k, n, 500 + b, kind="integer") for b in range(5)]
    As = [to_dev(a) for a, _ in ins]
    Bs = [to_dev(b) for _, b in ins]
    Cs = fmm.gemm_batched(p, As, Bs)
    torch.cuda.synchronize()
    for (A, B), C in zip(ins, Cs):
        assert np.array_equal(C.cpu().numpy(), oracle.gemm(A, B))
    if m % 2 ** levels == 0 and n % 2 ** levels == 0 and k % 2 ** levels == 0 and name == "strassen_222_7":
        # no fringe: one memset per product, then a single leaf launch for all products
        assert fmm.last_launch_count() == 1


FULL_SIZE = [
    # (algorithm, levels, precision, moduli, (m, k, n)): the benchmark's workloads
    ("strassen_222_7", 1, "ozaki_bf16", 12, (8192, 8192, 8192)),
    ("fmm_424_26", 3, "fp64", None, (8192, 8192, 8192)),
    ("fmm_333_23", 2, "fp64", None, (8192, 8192, 8192)),
    ("fmm_424_26", 1, "fp64", None, (16384, 2048, 16384)),
    ("strassen_222_7", 1, "ozaki_bf16", 12, (16384, 2048, 16384)),
    ("fmm_423_20", 1, "fp64", None, (16384, 2048, 2048)),
    ("fmm_323_15", 1, "ozaki_bf16", 12, (16384, 2048, 2048)),
]


@pytest.mark.parametrize("name,levels,precision,moduli,shape", FULL_SIZE)
def test_full_size_workloads_sampled(name, levels, precision, moduli, shape):
    # full-size products in the benchmark's launch configuration (level-by-
    # level scheme for FP64 plans, residue space for the emulated variant),
    # checked on sampled entries: within tolerance on uniform[-1,1], bit-exact
    # on the integer copy
    import torch
    m, k, n = shape
    flags = fmm.FLAG_LEVELWISE if precision == "fp64" else fmm.FLAGS_DEFAULT
    p = fmm.Plan(name, levels=levels, flags=flags, precision=precision, moduli=moduli)
    A, B = synth.operands(m, k, n, 1410)
    Ad, Bd = to_dev(A), to_dev(B)
    C = torch.empty((m, n), dtype=torch.float64, device="cuda")
    wsz = p.workspace_size(m, k, n)
    ws = torch.empty(wsz, dtype=torch.uint8, device="cuda") if wsz else None
    fmm.gemm(p, Ad, Bd, C=C, workspace=ws)
    torch.cuda.synchronize()
    fmm.check_device_error()
    rows, cols = synth.sample_indices(m, n, 512, 78)
    ri, ci = torch.from_numpy(rows).cuda(), torch.from_numpy(cols).cuda()
    e64, eld = oracle.gemm_entries(A, B, rows, cols)
    got = C[ri, ci].cpu().numpy()
    assert np.linalg.norm(got - eld) / np.linalg.norm(eld) <= TOL_F
    if precision == "ozaki_bf16":
        # the same scaled integers, their exact product and one rounding as
        # the oracle's emulation, entry by entry
        assert np.array_equal(got, ozaki.emulated_entries(A, B, rows, cols, moduli))
    Ai, Bi = np.rint(4 * A), np.rint(4 * B)
    Ad.copy_(torch.from_numpy(Ai))
    Bd.copy_(torch.from_numpy(Bi))
    fmm.gemm(p, Ad, Bd, C=C, workspace=ws)
    torch.cuda.synchronize()
    ei64, _ = oracle.gemm_entries(Ai, Bi, rows, cols)
    assert np.array_equal(C[ri, ci].cpu().numpy(), ei64)


def fast_abs_entries(name, A, B, rows, cols):
    """For a one-level plan: sum_r |W_qr| (|S_r| |T_r|)_ij at the sampled
    entries, |S_r| = sum_i |U_ir| |A_i| and |T_r| = sum_j |V_jr| |B_j| (block
    (i, j) of C in block q).  Leaf products with relative error e per term
    give C within e times this, entry by entry (the FP64 additions add
    rounding errors far below the bounds used)."""
    M, K, N, U, V, W = fmm.algorithm_factors(name)
    m, k = A.shape
    n = B.shape[1]
    mb, kb, nb = m // M, k // K, n // N
    out = np.zeros(len(rows))
    for t, (i, j) in enumerate(zip(rows, cols)):
        a, ii = divmod(int(i), mb)
        c, jj = divmod(int(j), nb)
        q = a * N + c
        for r in np.nonzero(W[q])[0]:
            srow = np.zeros(kb)
            for blk in np.nonzero(U[:, r])[0]:
                ba, bb = divmod(int(blk), K)
                srow += abs(U[blk, r]) * np.abs(A[ba * mb + ii, bb * kb:(bb + 1) * kb])
            tcol = np.zeros(kb)
            for blk in np.nonzero(V[:, r])[0]:
                bb, bc = divmod(int(blk), N)
                tcol += abs(V[blk, r]) * np.abs(B[bb * kb:(bb + 1) * kb, bc * nb + jj])
            out[t] += abs(W[q, r]) * float(srow @ tcol)
    return out


FULL_SIZE_PRECISION = [
    # (algorithm, levels, precision, moduli, (m, k, n), data): the precision
    # variants at the sizes the paper's largest square runs and the rank-k
    # workload use
    ("strassen_222_7", 1, "ozaki_bf16", 14, (16384, 16384, 16384), "uniform"),
    ("strassen_222_7", 1, "ozaki_bf16", 13, (16384, 16384, 16384), "loguniform"),
    ("fmm_424_26", 1, "ozaki_bf16", 14, (16384, 2048, 16384), "uniform"),
    ("strassen_222_7", 0, "tf32", None, (16384, 16384, 16384), "uniform"),
    ("strassen_222_7", 1, "tf32", None, (16384, 16384, 16384), "uniform"),
    ("strassen_222_7", 1, "fp32", None, (16384, 16384, 16384), "uniform"),
]


@pytest.mark.parametrize("name,levels,precision,moduli,shape,data", FULL_SIZE_PRECISION)
def test_full_size_precision_variants_sampled(name, levels, precision, moduli, shape, data):
    # emulated FP64: bit-identical to the oracle's emulation at every sampled
    # entry.  TF32 / FP32-accurate leaves: every sampled entry within its
    # rounding bound of the oracle's long-double value (k = 16384, the regime
    # where whole-k FP32 sums in the tensor core lose accuracy), and e_F within
    # the variant's stated error.
    import torch
    m, k, n = shape
    p = fmm.Plan(name, levels=levels, precision=precision, moduli=moduli)
    A, B = synth.operands(m, k, n, 1411, kind=data)
    Ad, Bd = to_dev(A), to_dev(B)
    C = torch.empty((m, n), dtype=torch.float64, device="cuda")
    wsz = p.workspace_size(m, k, n)
    ws = torch.empty(wsz, dtype=torch.uint8, device="cuda") if wsz else None
    fmm.gemm(p, Ad, Bd, C=C, workspace=ws)
    torch.cuda.synchronize()
    fmm.check_device_error()
    del ws
    rows, cols = synth.sample_indices(m, n, 256, 79)
    got = C[torch.from_numpy(rows).cuda(), torch.from_numpy(cols).cuda()].cpu().numpy()
    del Ad, Bd, C
    _, eld = oracle.gemm_entries(A, B, rows, cols)
    if precision == "ozaki_bf16":
        assert np.array_equal(got, ozaki.emulated_entries(A, B, rows, cols, moduli))
        # e_F: about 2^-beta on uniform data (beta = 47 for 14 moduli at
        # k = 16384); log-uniform rows lose the digits of their small entries
        # relative to the row maximum, so there the target is the plan's 1e-11
        assert np.linalg.norm(got - eld) / np.linalg.norm(eld) <= (2e-14 if data == "uniform" else TOL_F)
        return
    kL = k // 2 ** levels
    if levels == 0:
        _, absab = oracle.gemm_entries(np.abs(A), np.abs(B), rows, cols)
    else:
        absab = fast_abs_entries(name, A, B, rows, cols)
    if precision == "tf32":
        # operands rounded to FP32 then TF32 (2^-11 + 2^-24 each), FP32 sums
        # over the whole k in the tensor core (one unit in the last place per
        # addition at worst)
        factor = 2.0 ** -10 + 2.0 ** -20 + kL * 2.0 ** -23
        e_max = 1e-3
    else:
        # TF32 pairs keep 22 bits of each FP32 operand, lo x lo dropped; sums of
        # 512 k (x3 terms) in the tensor core, chunk sums added with round to
        # nearest on the CUDA cores
        factor = 4 * 2.0 ** -22 + 1.01 * 1536 * 2.0 ** -23 + (kL / 512 + 4) * 2.0 ** -24
        e_max = 1e-5
    assert np.all(np.abs(got - eld) <= factor * absab + 2.0 ** -40 * absab)
    assert np.linalg.norm(got - eld) / np.linalg.norm(eld) <= e_max
