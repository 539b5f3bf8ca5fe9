"""GPU checks of the mixed-precision path: FP32 vectors, vertex-patch solves
on tensor cores (tcgen05) in bf16 / fp16 with FP32 accumulation, FP64
iterative refinement outside (arXiv 2205.05840, eq. Preconditioner P, Fig. 1).

Tolerances are derived from the operand precision: a patch output is a sum
over 108 (then 60) products of rounded operands (r, W, then W^t r), each
rounding carrying a relative error of at most u = 2^-8 (bf16) or 2^-11
(fp16).  Measured against the largest entry the error is a few u for well
conditioned patches and grows with the patch condition (cond ~ alpha/h^2):
~10u at alpha/h^2 = 4e4; the tests allow 16u.  FP32 stencil / transfer results are held to
2e-6 relative.  Refined solves must reach the FP64 tolerance 1e-8 exactly as
the FP64 path does.
"""
import numpy as np
import scipy.linalg as sla
import pytest
import torch

from oracle import hcurl, mg
from paper_2205_05840_gb300 import inputs

pytestmark = pytest.mark.gpu

try:
    from paper_2205_05840_gb300 import ndmg
except ImportError:
    if torch.cuda.is_available():
        raise
    pytest.skip("library not built and no GPU here", allow_module_level=True)

DEV = "cuda"
U = {"bf16": 2.0 ** -8, "fp16": 2.0 ** -11}


def prec_code(p):
    return {"bf16": ndmg.PREC_MIXED_BF16, "fp16": ndmg.PREC_MIXED_FP16}[p]


def T(x, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device=DEV)


def N(t):
    torch.cuda.synchronize()
    return t.detach().double().cpu().numpy()


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


KERNELS = {"brick": 1, "cell": 2}


@pytest.mark.parametrize("kernel", ["brick", "cell"])
@pytest.mark.parametrize("prec", ["bf16", "fp16"])
@pytest.mark.parametrize("n,n0,alpha", [(4, 2, 1.0), (8, 4, 1.0), (12, 6, 0.01), (20, 10, 100.0), (32, 4, 1.0),
                                        (40, 5, 1.0)])
def test_tc_smoothing_step(kernel, prec, n, n0, alpha):
    # one smoothing step z <- z + M_V^{-1}(g - A z) on float vectors, patch
    # solves on tensor cores (both kernels), against the FP64 oracle (sizes:
    # one brick / column tile, several, partial ones)
    S = ndmg.Solver(n, n_coarsest=n0, alpha=alpha, precision=prec_code(prec))
    S.select_smoother(KERNELS[kernel])
    A = hcurl.assemble(n, 1.0, alpha, 1.0)
    Sm = mg.Smoother(A, n, "vertex")
    rng = np.random.default_rng(n)
    g = rng.standard_normal(A.shape[0]).astype(np.float32).astype(np.float64)
    z = rng.standard_normal(A.shape[0]).astype(np.float32).astype(np.float64)
    corr = Sm.apply(g - A @ z)
    zt = T(z)
    S.smooth(T(g), zt, steps=1, level=-1)
    got = N(zt) - z
    assert rel(got, corr) < 16 * U[prec]


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
@pytest.mark.parametrize("n,n0,alpha", [(4, 2, 1.0), (8, 4, 1.0), (12, 6, 0.01), (20, 10, 100.0), (32, 4, 1.0),
                                        (36, 9, 1.0), (40, 5, 1.0)])
def test_cuda_core_smoothing_step(prec, n, n0, alpha):
    # the FP32 CUDA-core smoother (one launch on levels with at most 4096
    # vertex patches, n <= 32 here; the staged pair above) against the FP64
    # oracle; FP32 arithmetic: sums of 108 products (relative 1e-5), and the
    # FP32-rounded patch operator, whose error grows with the patch matrix's
    # condition number (8 cond 2^-24, as the FP64 tests' bound with FP64 eps)
    code = ndmg.PREC_FP32 if prec == "fp32" else ndmg.PREC_MIXED_FP16
    S = ndmg.Solver(n, n_coarsest=n0, alpha=alpha, precision=code)
    S.select_smoother(0)
    A = hcurl.assemble(n, 1.0, alpha, 1.0)
    Sm = mg.Smoother(A, n, "vertex")
    rng = np.random.default_rng(n + 1)
    g = rng.standard_normal(A.shape[0]).astype(np.float32).astype(np.float64)
    z = rng.standard_normal(A.shape[0]).astype(np.float32).astype(np.float64)
    corr = Sm.apply(g - A @ z)
    zt = T(z)
    S.smooth(T(g), zt, steps=1, level=-1)
    got = N(zt) - z
    kappa = np.linalg.cond(hcurl.assemble(4, 4.0 / n, alpha, 1.0).toarray())
    assert rel(got, corr) < max(1e-5, 8 * kappa * 2.0 ** -24)


@pytest.mark.parametrize("kernel", ["brick", "cell"])
@pytest.mark.parametrize("prec", ["bf16", "fp16"])
@pytest.mark.parametrize("n", [64, 128])
def test_tc_smoothing_step_sampled_cells(kernel, prec, n):
    # one tensor-core smoothing step at 64^3 and 128^3 against the oracle on
    # every edge of sampled coarse cells: the domain faces, the borders of the
    # kernel's 14-cell column tiles (13|14, 27|28, ...) and random cells.  The
    # oracle's patch and interior operators come from an 8^3 grid with the same
    # h (every interior patch matrix is the same), the residual from its
    # element-by-element rows
    nc = n // 2
    h = 1.0 / n
    S = ndmg.Solver(n, n_coarsest=4, precision=prec_code(prec))
    S.select_smoother(KERNELS[kernel])
    rng = np.random.default_rng(n + 1)
    Nn = hcurl.num_edges(n)
    g = rng.standard_normal(Nn).astype(np.float32).astype(np.float64)
    z = rng.standard_normal(Nn).astype(np.float32).astype(np.float64)
    zt = T(z)
    S.smooth(T(g), zt, steps=1, level=-1)
    got = N(zt) - z
    small = mg.Smoother(hcurl.assemble(8, 8 * h, 1.0, 1.0), 8, "vertex")
    (pidx8, patch), = small.patches
    cT = small.cT
    # local numbering of a patch / interior space: the small grid's first
    # patch and block, shifted to the vertex / cell of interest
    d8, i8, j8, k8 = hcurl.edge_coords_of(8, pidx8[0])
    bub8 = mg.bubble_sets(8)[0]
    db, ib, jb, kb = hcurl.edge_coords_of(8, bub8)
    edges_of = lambda d, i, j, k: hcurl.edge_index(n, d, i, j, k)
    border = sorted({0, 1, nc - 2, nc - 1} | {c for q in range(1, nc // 14 + 1) for c in (14 * q - 1, 14 * q)
                                              if c < nc})
    cells = [(cx, cy, cz) for cx in border[::2] for cy in border[1::2] for cz in (0, nc // 2, nc - 1)]
    cells += [tuple(rng.integers(0, nc, 3)) for _ in range(12)]
    want, have = [], []
    for (cx, cy, cz) in cells:
        own = {}
        for d in range(3):
            for c in range(2):
                for b in range(2):
                    for a in range(2):
                        e = edges_of(d, 2 * cx + a, 2 * cy + b, 2 * cz + c)
                        if e >= 0:
                            own[int(e)] = 0.0
        keys = np.array(list(own))
        # vertex patches containing the cell's edges: V in C + {0, 1}^3, interior
        for V in [(cx + a, cy + b, cz + c) for c in range(2) for b in range(2) for a in range(2)]:
            if min(V) < 1 or max(V) > nc - 1:
                continue
            sh = 2 * (np.array(V) - 1)   # the small grid's first patch sits at vertex (1, 1, 1)
            rows = edges_of(d8, i8 + sh[0], j8 + sh[1], k8 + sh[2])
            rv = g[rows] - hcurl.apply_rows(n, 1.0, 1.0, 1.0, z, rows)
            y = patch.apply(rv[:, None])[:, 0]
            for e, val in zip(rows, y):
                if int(e) in own:
                    own[int(e)] += val
        # interior space of the cell itself
        rows = edges_of(db, ib + 2 * cx, jb + 2 * cy, kb + 2 * cz)
        rv = g[rows] - hcurl.apply_rows(n, 1.0, 1.0, 1.0, z, rows)
        for e, val in zip(rows, sla.cho_solve(cT, rv)):
            own[int(e)] += val
        want.extend(small.eta * own[int(e)] for e in keys)
        have.extend(got[keys])
    want, have = np.array(want), np.array(have)
    assert rel(have, want) < 16 * U[prec]


@pytest.mark.parametrize("kernel", ["brick", "cell"])
@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_tc_patch_columns(kernel, prec):
    # a unit residual on single edges: the correction is one column of the
    # smoother (every patch index must land on the right edge)
    n = 12
    S = ndmg.Solver(n, n_coarsest=6, precision=prec_code(prec))
    S.select_smoother(KERNELS[kernel])
    A = hcurl.assemble(n, 1.0, 1.0, 1.0)
    Sm = mg.Smoother(A, n, "vertex")
    Nn = A.shape[0]
    # g = A z + e_j  =>  residual = e_j exactly (FP32 stencil on z = 0)
    for j in (0, 17, Nn // 3, Nn // 2 + 5, Nn - 1, hcurl.edge_index(n, 1, 5, 6, 7), hcurl.edge_index(n, 2, 6, 6, 6)):
        g = np.zeros(Nn)
        g[j] = 1.0
        zt = torch.zeros(Nn, dtype=torch.float32, device=DEV)
        S.smooth(T(g), zt, steps=1)
        col = Sm.apply(g)
        got = N(zt)
        assert rel(got, col) < 16 * U[prec], j
        assert set(np.nonzero(np.abs(got) > 1e-3 * np.abs(col).max())[0]) <= set(np.nonzero(col)[0])


@pytest.mark.parametrize("small", ["persistent", "separate"])
@pytest.mark.parametrize("kernel", ["brick", "cell"])
@pytest.mark.parametrize("prec", ["bf16", "fp16"])
@pytest.mark.parametrize("n,n0", [(16, 2), (32, 4), (24, 3), (64, 4)])
def test_mixed_vcycle_close_to_oracle(small, kernel, prec, n, n0):
    # the levels <= 16^3 below the finest in one cluster launch (FP32 CUDA
    # cores) or in separate launches (tensor-core smoother)
    S = ndmg.Solver(n, n_coarsest=n0, precision=prec_code(prec))
    S.select_smoother(KERNELS[kernel])
    S.select_smoother(1 if small == "persistent" else 0, level=0)
    H = mg.Hierarchy(n, 1.0, 1.0, 1.0, n0=n0, m=2)
    f = inputs.random_load(n, 0)
    ref = H.vcycle(f, np.zeros_like(f))
    zt = torch.zeros(f.size, dtype=torch.float32, device=DEV)
    S.vcycle(T(f), zt)
    # one V-cycle is a product of ~(4m+1)*levels rounded operators; the
    # deviation from the FP64 cycle stays within 16u of the result's size
    assert rel(N(zt), ref) < 16 * U[prec]


@pytest.mark.parametrize("method", ["pcg", "ir"])
@pytest.mark.parametrize("prec", ["bf16", "fp16", "fp32"])
@pytest.mark.parametrize("n,n0,alpha", [(32, 4, 1.0), (64, 4, 0.01), (48, 3, 100.0)])
def test_mixed_refined_solve_reaches_fp64_tolerance(method, prec, n, n0, alpha):
    # FP64 PCG with the low-precision V-cycle as preconditioner, and FP64
    # iterative refinement around a float PCG: both reach the FP64 tolerance
    code = ndmg.PREC_FP32 if prec == "fp32" else prec_code(prec)
    S = ndmg.Solver(n, n_coarsest=n0, alpha=alpha, precision=code)
    f = inputs.random_load(n, 4)
    u = torch.zeros(f.size, dtype=torch.float64, device=DEV)
    if method == "pcg":
        st, it, rr = S.solve(T(f, torch.float64), u, tol=1e-8, maxit=300)
    else:
        st, it, rr = S.solve_ir(T(f, torch.float64), u, tol=1e-8, inner_tol=1e-4, maxit=300)
    assert rr <= 1e-8
    # independent FP64 check of the residual, then against the FP64 GPU solve
    S64 = ndmg.Solver(n, n_coarsest=n0, alpha=alpha)
    r = torch.empty_like(u)
    S64.residual(T(f, torch.float64), u, r)
    assert np.linalg.norm(N(r)) / np.linalg.norm(f) <= 1.01e-8
    u64 = torch.zeros_like(u)
    S64.solve(T(f, torch.float64), u64, tol=1e-10)
    assert rel(N(u), N(u64)) < 1e-6


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_mixed_128_full_size(prec):
    # the benchmark configuration: 128^3, alpha = 1, seed-0 load, coarsest 4^3
    n = 128
    S = ndmg.Solver(n, n_coarsest=4, precision=prec_code(prec))
    f = inputs.random_load(n, 0)
    ft = T(f, torch.float64)
    u = torch.zeros(f.size, dtype=torch.float64, device=DEV)
    st, it, rr = S.solve(ft, u, tol=1e-8, maxit=300)
    assert rr <= 1e-8 and it < 60
    S64 = ndmg.Solver(n, n_coarsest=4)
    r = torch.empty_like(u)
    S64.residual(ft, u, r)
    assert np.linalg.norm(N(r)) / np.linalg.norm(f) <= 1.01e-8
    # sampled rows of the operator in FP32 against the oracle
    x = np.random.default_rng(3).standard_normal(f.size).astype(np.float32)
    y = torch.empty(f.size, dtype=torch.float32, device=DEV)
    S.apply(T(x), y)
    rows = np.random.default_rng(4).integers(0, f.size, 2000)
    ref = hcurl.apply_rows(n, 1.0, 1.0, 1.0, x.astype(np.float64), rows)
    assert rel(N(y)[rows], ref) < 2e-6


def test_mixed_manufactured_64():
    n, alpha = 64, 1.0
    h = 1.0 / n
    S = ndmg.Solver(n, n_coarsest=4, alpha=alpha, precision=ndmg.PREC_MIXED_BF16)
    f = inputs.manufactured_load(n, 1.0, alpha, 1.0)
    u = torch.zeros(f.size, dtype=torch.float64, device=DEV)
    st, it, rr = S.solve(T(f, torch.float64), u, tol=1e-8)
    mu = (2.0 + np.cos(np.pi * h)) / 3.0
    sig = (np.sin(np.pi * h / 2) / (np.pi * h / 2)) ** 2
    c = (2 * np.pi ** 2 * alpha + 1) * sig ** 2 / (8 * alpha * np.sin(np.pi * h / 2) ** 2 * mu / h ** 2 + mu ** 2)
    assert rr <= 1e-8 and rel(N(u), c * inputs.sine_interpolant(n)) < 1e-6


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_graph_replay_matches_direct_launches(prec):
    # the mixed solve replays its float V-cycle as a CUDA graph; direct
    # launches give the same iteration count and launch / V-cycle counters,
    # solutions agree to the solve tolerance (FP32 atomics make the last bits
    # run-dependent), and traced kernel times are collected from the replays.
    # 64^3: the finest levels smooth on tensor cores, the levels <= 16^3 run in
    # the small-level cluster kernel (one launch per V-cycle, traced too)
    n = 64
    f = torch.tensor(inputs.random_load(n, 3), dtype=torch.float64, device=DEV)
    out = {}
    for graphs in (False, True):
        S = ndmg.Solver(n, n_coarsest=4, precision=prec_code(prec))
        S.select_smoother(1, level=0)          # the levels <= 16^3 in one cluster launch
        S.use_graphs(graphs)
        S.trace(ndmg.K_PATCH, True)
        S.trace(ndmg.K_COARSE, True)
        S.trace_read(ndmg.K_PATCH)
        S.trace_read(ndmg.K_COARSE)
        u = torch.zeros_like(f)
        l0, v0 = S.counters()
        st, it, rr = S.solve(f, u, tol=1e-10)
        l1, v1 = S.counters()
        n_l, ms, units = S.trace_read(ndmg.K_PATCH)
        n_c, ms_c, _ = S.trace_read(ndmg.K_COARSE)
        assert rr <= 1e-10 and n_l > 0 and ms > 0 and units > 0
        assert n_c == v1 - v0 and ms_c > 0            # one small-level launch per V-cycle
        out[graphs] = (it, l1 - l0, v1 - v0, n_l, units, u.cpu().numpy())
    a, b = out[False], out[True]
    assert abs(a[0] - b[0]) <= 1                      # iterations (last-bit effects only)
    assert a[1] * b[2] == b[1] * a[2]                  # launches per V-cycle
    assert a[3] * b[2] == b[3] * a[2] and abs(a[4] / a[3] - b[4] / b[3]) < 1e-9 * a[4] / a[3]
    assert np.linalg.norm(a[5] - b[5]) <= 1e-8 * np.linalg.norm(a[5])


def test_bf16_rejects_operator_it_cannot_represent():
    # alpha / (beta h^2) = 4.1e5 (alpha = 100 at 64^3): the bf16-rounded Gram
    # factor gives A_p W~W~^t an eigenvalue of 23 instead of 1 and the solve
    # diverged; the library refuses it at set-up and fp16 handles the case
    with pytest.raises(ndmg.NdmgError) as e:
        ndmg.Solver(64, n_coarsest=4, alpha=100.0, precision=ndmg.PREC_MIXED_BF16)
    assert e.value.status == ndmg.INVALID_ARG
    f = T(inputs.random_load(64, 0), torch.float64)
    S = ndmg.Solver(64, n_coarsest=4, alpha=1.0, precision=ndmg.PREC_MIXED_BF16)
    with pytest.raises(ndmg.NdmgError):
        S.set_alpha(100.0)
    u = torch.zeros_like(f)
    st, it, rr = S.solve(f, u, tol=1e-8)          # still the alpha = 1 operators
    assert rr <= 1e-8
    S16 = ndmg.Solver(64, n_coarsest=4, alpha=100.0, precision=ndmg.PREC_MIXED_FP16)
    u = torch.zeros_like(f)
    st, it, rr = S16.solve(f, u, tol=1e-8)
    assert rr <= 1e-8


def test_autotune_changes_launch_shapes_not_results():
    # ndmg_autotune picks the stencil's z-planes per CTA per level by timing;
    # every choice computes the same values, bit for bit
    n = 64
    S = ndmg.Solver(n, n_coarsest=4, precision=ndmg.PREC_MIXED_FP16)
    rng = np.random.default_rng(5)
    res = {}
    for dt in (torch.float32, torch.float64):
        for lv in range(S.num_levels):
            Nl = S.num_dofs(lv)
            x, g = T(rng.standard_normal(Nl), dt), T(rng.standard_normal(Nl), dt)
            r = torch.empty_like(x)
            S.residual(g, x, r, level=lv)
            res[(dt, lv)] = (x, g, N(r))
    f = T(inputs.random_load(n, 0), torch.float64)
    u = torch.zeros_like(f)
    _, it0, _ = S.solve(f, u, tol=1e-8)
    choices = S.autotune()
    assert set(choices) == set(range(S.num_levels))
    for lv, (cf, cd, tc) in choices.items():
        nl = 4 << lv
        for c in (cf, cd):
            assert c >= 1 and c <= nl and (c & (c - 1)) == 0
        # 0: CUDA-core smoother, 1: tensor cores per brick, 2: cell-owned rows;
        # level 0 (no smoother): 1 when the levels <= 16^3 run in one launch
        assert tc in (0, 1, 2) and (lv > 0 or tc in (0, 1))
    for (dt, lv), (x, g, r0) in res.items():
        r = torch.empty_like(x)
        S.residual(g, x, r, level=lv)
        assert np.array_equal(N(r), r0), (dt, lv)
    u = torch.zeros_like(f)
    _, it1, rr = S.solve(f, u, tol=1e-8)
    assert rr <= 1e-8 and abs(it1 - it0) <= 2
    # whatever smoother each level got, one smoothing step still matches the oracle
    A = hcurl.assemble(n, 1.0, 1.0, 1.0)
    Sm = mg.Smoother(A, n, "vertex")
    g = rng.standard_normal(A.shape[0]).astype(np.float32).astype(np.float64)
    zt = torch.zeros(A.shape[0], dtype=torch.float32, device=DEV)
    S.smooth(T(g), zt, steps=1)
    assert rel(N(zt), Sm.apply(g)) < 16 * U["fp16"]


@pytest.mark.gpu
def test_set_launch_shapes_reproduces_autotuned_handle():
    # ndmg_set_launch_shapes applies ndmg_autotune's choices to another handle
    # without timing: the same V-cycle count, solutions within the float
    # V-cycle's summation-order noise, and every entry checked before use
    n = 64
    f = T(inputs.random_load(n, 0), torch.float64)
    S1 = ndmg.Solver(n, n_coarsest=4, precision=ndmg.PREC_MIXED_FP16)
    tuned = S1.autotune()
    u1 = torch.zeros_like(f)
    _, it1, rr1 = S1.solve(f, u1, tol=1e-8)
    S2 = ndmg.Solver(n, n_coarsest=4, precision=ndmg.PREC_MIXED_FP16)
    S2.set_launch_shapes(tuned)
    u2 = torch.zeros_like(f)
    _, it2, rr2 = S2.solve(f, u2, tol=1e-8)
    assert rr1 <= 1e-8 and rr2 <= 1e-8 and it1 == it2
    assert rel(N(u2), N(u1)) < 1e-7
    # the other way round: every smoother forced, then applied by hand
    forced = {k: (1, 1, 0 if k == 0 else 2) for k in tuned}
    S2.set_launch_shapes(forced)
    u2.zero_()
    _, it3, rr3 = S2.solve(f, u2, tol=1e-8)
    assert rr3 <= 1e-8 and abs(it3 - it1) <= 2
    bad = dict(tuned)
    bad[S2.num_levels - 1] = (n + 1, 1, 1)      # more planes per CTA than the level has
    with pytest.raises(ndmg.NdmgError):
        S2.set_launch_shapes(bad)
    bad = dict(tuned)
    bad[1] = (1, 1, 3)                          # no smoother kind 3
    with pytest.raises(ndmg.NdmgError):
        S2.set_launch_shapes(bad)
    S64 = ndmg.Solver(16, n_coarsest=4)
    with pytest.raises(ndmg.NdmgError):          # tensor-core smoothers need a MIXED handle
        S64.set_launch_shapes({0: (1, 1, 0), 1: (1, 1, 1), 2: (1, 1, 0)})


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_mixed_solve_takes_the_fp64_vcycle_count(prec):
    # the tensor-core smoother forms its patch outputs with W's high and
    # low-order parts: a single rounding of W there costs V-cycles (fp16:
    # 17 against 15 at 128^3, bf16: 22), the other roundings do not, so the
    # mixed solve needs (about) the FP64 V-cycle's iterations
    n = 64
    f = T(inputs.random_load(n, 0), torch.float64)
    S64 = ndmg.Solver(n, n_coarsest=4)
    u = torch.zeros_like(f)
    _, it64, _ = S64.solve(f, u, tol=1e-8)
    S = ndmg.Solver(n, n_coarsest=4, precision=prec_code(prec))
    S.select_smoother(1)
    u.zero_()
    _, it, rr = S.solve(f, u, tol=1e-8)
    assert rr <= 1e-8 and it <= it64 + 1, (it, it64)
