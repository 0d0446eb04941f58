"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Error measure: rel = max_i |H_gpu,i - H_ref,i|_2 / max_i |H_ref,i|_2 over macro
points i. Bounds: 1e-12 for the FP64 method, 1e-6 for the batched FP32 form
(the accuracy targets stated for the two forms).

The FP64 method is compared with the oracle evaluated in long double: the
oracle's own FP64 rounding floor for H_avg is 1-3e-12 relative (measured in
tests/test_oracle_precision.py), above the 1e-12 bar, so a long-double
evaluation of the same scheme is the reference that can resolve it. The FP32
form is compared with the FP64 oracle.

Small cases run the oracle on every box; full-size workloads run the GPU on the
whole batch (the launch configuration the benchmark times) and the oracle on a
sample of boxes, including the largest and smallest boxes of uneven batches.
"""
import numpy as np
import pytest

import workloads as W
from oracle import hmm_oracle as O

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-6}
ORACLE_FP64_FLOOR = 3e-12      # bound on the FP64 oracle's own rounding error (relative)
N_LD_POINTS = 6                # boxes evaluated by the long-double oracle per case


def reference(cfg, M0, precision, points=None):
    """Oracle H_avg at ``points`` (FP64 oracle for the FP32 form, long double for FP64)."""
    if precision == 0:
        if points is None:
            P = cfg.n_points
            points = sorted(set([0, P - 1] + list(range(0, P, max(1, P // (N_LD_POINTS - 2))))))[:N_LD_POINTS]
        H = O.micro_batch(cfg, M0, points=points, dtype=np.longdouble)
        return points, H
    return points, O.micro_batch(cfg, M0, points=points)


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_09463_gb300 import build
    build()
    return torch


def rel_err(Hg, Hr):
    d = (np.asarray(Hg, dtype=Hr.dtype) - Hr).astype(np.float64)
    return np.linalg.norm(d, axis=0).max() / np.linalg.norm(Hr.astype(np.float64), axis=0).max()


def gpu_micro(torch, cfg, M0, precision, kernel_variant=0):
    from paper_2108_09463_gb300 import HMM
    h = HMM(cfg, precision=precision, kernel_variant=kernel_variant)
    M = torch.from_numpy(M0).cuda()
    H = h.micro_batch(M).cpu().numpy()
    info = h.box_info()
    h.close()
    return H, info


SMALL = {
    "c1_full": ("c1_1d", {}),
    "1d_order2_interp2": ("c1_1d", dict(n_macro=(16, 1, 1), box_n=81, micro_steps=120,
                                        stencil_order=2, interp_order=2)),
    "2d_small": ("c2_2d", dict(n_macro=(8, 8, 1), box_n=24, micro_steps=60)),
    "2d_ragged": ("c2_2d", dict(n_macro=(6, 7, 1), box_n=37, micro_steps=33)),
    "2d_order2": ("c2_2d", dict(n_macro=(8, 8, 1), box_n=24, micro_steps=50, stencil_order=2)),
    "3d_small": ("c4_3d", dict(n_macro=(5, 5, 6), box_n=16, mu_over_eps=0.9, micro_steps=30)),
    "2d_slow_fast": ("c3_2d_uneven", dict(n_macro=(8, 8, 1), eps_field=None, box_n_field=None,
                                          eps=1 / 250, box_n=32, micro_steps=40)),
}


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32"])
@pytest.mark.parametrize("case", sorted(SMALL))
def test_small_parity(torch_cuda, case, precision):
    name, over = SMALL[case]
    cfg = W.config(name, **over)
    if name == "c3_2d_uneven":
        cfg = cfg.replace(eps_field=None, box_n_field=None)
    M0 = W.initial_field(cfg)
    Hg, info = gpu_micro(torch_cuda, cfg, M0, precision)
    pts, Hr = reference(cfg, M0, precision)
    e = rel_err(Hg if pts is None else Hg[:, pts], Hr)
    assert e < TOL[precision], (case, precision, e)
    # the library's per-box geometry equals the oracle's
    for p in (0, cfg.n_points - 1):
        geo = O.box_geometry(cfg, p)
        assert info["N"][p] == geo["N"]
        assert abs(info["dt"][p] / geo["dt"] - 1) < 1e-14
        assert abs(info["mu"][p] / geo["mu"] - 1) < 1e-14


# Edge sizes: the smallest boxes (one interior node pair per axis, N = 2r + 2, with the
# averaging box [-mu, mu] shrunk inside the interior), the fewest micro steps that give
# a non-zero time average (M = 2: w_1 = 1), and the largest box per dimension that
# hmm_init accepts (N = 1024 / 256 / 64 for d = 1 / 2 / 3).
EDGE = {
    "2d_min_box_order4": ("c2_2d", dict(n_macro=(6, 5, 1), box_n=8, mu_over_eps=0.15, micro_steps=30)),
    "2d_min_box_order2": ("c2_2d", dict(n_macro=(6, 5, 1), box_n=4, stencil_order=2, mu_over_eps=0.15,
                                        micro_steps=30)),
    "2d_two_micro_steps": ("c2_2d", dict(n_macro=(6, 6, 1), box_n=24, micro_steps=2)),
    "1d_max_box": ("c1_1d", dict(n_macro=(8, 1, 1), box_n=1024, micro_steps=20)),
    "2d_max_box": ("c2_2d", dict(n_macro=(5, 5, 1), box_n=256, micro_steps=8)),
    "3d_max_box": ("c4_3d", dict(n_macro=(5, 5, 5), box_n=64, micro_steps=4)),
}


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32"])
@pytest.mark.parametrize("case", sorted(EDGE))
def test_edge_sizes_parity(torch_cuda, case, precision):
    name, over = EDGE[case]
    cfg = W.config(name, **over)
    M0 = W.initial_field(cfg)
    Hg, info = gpu_micro(torch_cuda, cfg, M0, precision)
    assert np.all(np.isfinite(Hg))
    P = cfg.n_points
    pts = sorted(set([0, P // 2, P - 1]))
    _, Hr = reference(cfg, M0, precision, points=pts)
    e = rel_err(Hg[:, pts], Hr)
    assert e < TOL[precision], (case, precision, e)
    assert info["N"][0] == O.box_geometry(cfg, 0)["N"]


# The RK4P micro stepper (Section 3.1) on the generic kernels, both precisions.
RK4P = {
    "1d": ("c1_1d", dict(n_macro=(16, 1, 1), box_n=81, micro_steps=60, micro_stepper=1)),
    "2d": ("c2_2d", dict(n_macro=(8, 8, 1), box_n=24, micro_steps=40, micro_stepper=1)),
    "2d_low_damping": ("c5_sweep", dict(n_macro=(8, 8, 1), box_n=32, micro_steps=40, alpha_micro=0.01,
                                        micro_stepper=1)),
    "3d": ("c4_3d", dict(n_macro=(5, 5, 6), box_n=16, mu_over_eps=0.9, micro_steps=20, micro_stepper=1)),
}


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32"])
@pytest.mark.parametrize("case", sorted(RK4P))
def test_rk4p_parity(torch_cuda, case, precision):
    name, over = RK4P[case]
    cfg = W.config(name, **over)
    M0 = W.initial_field(cfg)
    Hg, info = gpu_micro(torch_cuda, cfg, M0, precision)
    pts, Hr = reference(cfg, M0, precision)
    e = rel_err(Hg if pts is None else Hg[:, pts], Hr)
    assert e < TOL[precision], (case, precision, e)
    geo = O.box_geometry(cfg, 0)
    assert abs(info["dt"][0] / geo["dt"] - 1) < 1e-12   # the RK4P stability limit, host vs oracle


# RK4P on the resident 2D kernel (its own instances: a third state array and the
# per-node stage accumulator); 3D RK4P runs on the generic kernel.
RK4P_RESIDENT = {
    "pack_n24": ("c2_2d", dict(n_macro=(8, 8, 1), box_n=24, micro_steps=40, micro_stepper=1)),
    "low_damping_n32": ("c5_sweep", dict(n_macro=(8, 8, 1), box_n=32, micro_steps=40, alpha_micro=0.01,
                                         micro_stepper=1)),
    "ragged_n37": ("c2_2d", dict(n_macro=(6, 7, 1), box_n=37, micro_steps=24, micro_stepper=1)),
    "cluster_n64": ("c2_2d", dict(n_macro=(6, 6, 1), box_n=64, micro_steps=30, micro_stepper=1)),
    "cluster_n96": ("c5_sweep", dict(n_macro=(5, 5, 1), box_n=96, micro_steps=20, alpha_micro=0.1,
                                     micro_stepper=1)),
    "order2": ("c2_2d", dict(n_macro=(8, 8, 1), box_n=24, micro_steps=40, stencil_order=2, micro_stepper=1)),
}


@pytest.mark.parametrize("case", sorted(RK4P_RESIDENT))
def test_rk4p_resident_2d(torch_cuda, case):
    name, over = RK4P_RESIDENT[case]
    cfg = W.config(name, **over)
    M0 = W.initial_field(cfg)
    Hg, info = gpu_micro(torch_cuda, cfg, M0, 1, kernel_variant=2)
    pts = sorted(set([0, cfg.n_points // 2, cfg.n_points - 1]))
    Hr = O.micro_batch(cfg, M0, points=pts)
    assert rel_err(Hg[:, pts], Hr) < TOL[1], (case, rel_err(Hg[:, pts], Hr))


# The multi-step micro steppers MPE (2) and MPEA (3) on the generic kernels, both
# precisions: RK4P start-up steps, then the midpoint update with extrapolated h
# (Section 3.1); their time step from the AB2/AB3 stability regions (Section 3.2).
MULTISTEP = {
    "mpea_1d": ("c1_1d", dict(n_macro=(16, 1, 1), box_n=81, micro_steps=120, alpha_micro=0.1, micro_stepper=3)),
    "mpe_2d": ("c2_2d", dict(n_macro=(6, 5, 1), box_n=24, micro_steps=60, micro_stepper=2)),
    "mpea_2d_low_damping": ("c5_sweep", dict(n_macro=(6, 6, 1), box_n=48, micro_steps=60, alpha_micro=0.01,
                                             micro_stepper=3)),
    "mpea_2d_order2": ("c2_2d", dict(n_macro=(6, 5, 1), box_n=25, micro_steps=50, stencil_order=2, micro_stepper=3)),
    "mpea_3d": ("c4_3d", dict(n_macro=(5, 5, 5), box_n=16, mu_over_eps=0.9, micro_steps=30, micro_stepper=3)),
    "mpea_startup_only": ("c2_2d", dict(n_macro=(6, 5, 1), box_n=24, micro_steps=2, micro_stepper=3)),
    "mpe_three_steps": ("c2_2d", dict(n_macro=(6, 5, 1), box_n=24, micro_steps=3, micro_stepper=2)),
}


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32"])
@pytest.mark.parametrize("case", sorted(MULTISTEP))
def test_multistep_micro_steppers(torch_cuda, case, precision):
    name, over = MULTISTEP[case]
    cfg = W.config(name, **over)
    M0 = W.initial_field(cfg)
    Hg, info = gpu_micro(torch_cuda, cfg, M0, precision)
    pts = sorted(set([0, 1, cfg.n_points // 2, cfg.n_points - 1]))
    Hr = O.micro_batch(cfg, M0, points=pts, dtype=np.longdouble if precision == 0 else np.float64)
    e = rel_err(Hg[:, pts], Hr)
    assert e < TOL[precision], (case, precision, e)
    for p in (0, cfg.n_points - 1):
        geo = O.box_geometry(cfg, p)
        assert abs(info["dt"][p] / geo["dt"] - 1) < 1e-12   # the AB2/AB3 stability rule, host vs oracle


def test_multistep_not_resident(torch_cuda):
    from paper_2108_09463_gb300 import HMM, HmmError
    cfg = W.config("c2_2d", n_macro=(5, 5, 1), box_n=32, micro_steps=10, micro_stepper=3)
    with pytest.raises(HmmError) as ei:
        HMM(cfg, precision=1, kernel_variant=2)
    assert ei.value.status == 1


def test_rk4p_3d_not_resident(torch_cuda):
    from paper_2108_09463_gb300 import HMM, HmmError
    cfg = W.config("c4_3d", n_macro=(5, 5, 5), box_n=32, micro_steps=10, micro_stepper=1)
    with pytest.raises(HmmError) as ei:
        HMM(cfg, precision=1, kernel_variant=2)
    assert ei.value.status == 1


# Coefficients that are not sums of separable terms, tabulated at the faces
# (hmm_set_face_table): the locally periodic 2D example of Section 5 and a 1D one.
TABLE = {
    "loc2d": ("ex_loc2d", dict(n_macro=(6, 5, 1), box_n=29, mu_over_eps=0.0, micro_steps=40)),
    # a 3D box the z-column kernel would take: the table moves it to the z-slab kernel
    "3d_n32": ("c4_3d", dict(n_macro=(5, 5, 5), box_n=32, micro_steps=12,
                             coef_fn=lambda X, eps: 1.0 + 0.5 * np.sin(2 * np.pi * X[0] / eps)
                             * np.sin(2 * np.pi * X[1] / eps) * np.cos(2 * np.pi * X[2] / eps + 0.3))),
    "loc1d": ("c1_1d", dict(n_macro=(16, 1, 1), box_n=81, micro_steps=60,
                            coef_fn=lambda X, eps: 1.1 + 0.25 * np.sin(2 * np.pi * X[0] + 1.1)
                            + 0.5 * np.sin(2 * np.pi * X[0] / eps))),
}


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32"])
@pytest.mark.parametrize("case", sorted(TABLE))
def test_face_table_parity(torch_cuda, case, precision):
    from paper_2108_09463_gb300 import HMM
    name, over = TABLE[case]
    cfg = W.config(name, **over)
    M0 = W.initial_field(cfg)
    h = HMM(cfg, precision=precision, face_table=W.face_table(cfg))
    Hg = h.micro_batch(torch_cuda.from_numpy(M0).cuda()).cpu().numpy()
    info = h.box_info()
    assert abs(h.macro_dt() / O.macro_dt(cfg) - 1) < 1e-12
    h.close()
    for p in (0, cfg.n_points - 1):   # the micro step from each box's own maximum
        assert abs(info["dt"][p] / O.box_geometry(cfg, p)["dt"] - 1) < 1e-12
    pts, Hr = reference(cfg, M0, precision)
    e = rel_err(Hg if pts is None else Hg[:, pts], Hr)
    assert e < TOL[precision], (case, precision, e)


def test_face_table_rejects_bad_tables(torch_cuda):
    from paper_2108_09463_gb300 import HMM, HmmError
    cfg = W.config("ex_loc2d", n_macro=(6, 5, 1), box_n=29, mu_over_eps=0.0, micro_steps=10)
    tab = W.face_table(cfg)
    h = HMM(cfg, precision=1)
    with pytest.raises(HmmError):
        h.set_face_table(tab[:-1])          # wrong length
    bad = tab.copy()
    bad[5] = -1.0                           # a used face of box 0, axis 0: (A1)
    with pytest.raises(HmmError):
        h.set_face_table(bad)
    h.close()


def _uneven_small():
    cfg = W.config("c3_2d_uneven", n_macro=(12, 12, 1), micro_steps=40, eps_field=None, box_n_field=None)
    eps, n = W.uneven_eps_and_n(cfg, K=8.0, mu_prime=0.0075, nmin=24, nmax=48, step=8)
    return cfg.replace(eps_field=eps, box_n_field=n)


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32"])
def test_uneven_boxes_parity(torch_cuda, precision):
    cfg = _uneven_small()
    M0 = W.initial_field(cfg)
    Hg, info = gpu_micro(torch_cuda, cfg, M0, precision)
    N = info["N"]
    assert N.min() == 24 and N.max() == 48
    nsample = 4 if precision == 0 else 14
    pts = sorted(set([int(np.argmin(N)), int(np.argmax(N))] +
                     list(np.random.default_rng(0).choice(cfg.n_points, nsample, replace=False))))
    _, Hr = reference(cfg, M0, precision, pts)
    assert rel_err(Hg[:, pts], Hr) < TOL[precision]


RESIDENT_2D = ["2d_small", "2d_ragged", "2d_order2", "2d_slow_fast"]

# Row groups of 16 or 32 tiles with two lanes of slack take the right-hand y faces
# from the next lanes by shuffles: odd interior widths (the tile's second column is
# ring), both stencil orders, the two-lane slack exactly (Ni = 28 and 60 on the box-
# stride instance, when the plan picks it), a cluster of CTAs and RK4P.
YSHFL = {
    "canvas64_odd_n63": ("c2_2d", dict(n_macro=(5, 6, 1), box_n=63, micro_steps=30)),
    "order2_odd_n27": ("c2_2d", dict(n_macro=(6, 5, 1), box_n=27, micro_steps=40, stencil_order=2)),
    "slack2_n34": ("c2_2d", dict(n_macro=(6, 5, 1), box_n=34, micro_steps=30)),
    "slack2_n66": ("c2_2d", dict(n_macro=(5, 5, 1), box_n=66, micro_steps=24)),
    "rk4p_n63": ("c2_2d", dict(n_macro=(5, 5, 1), box_n=63, micro_steps=24, micro_stepper=1)),
}


@pytest.mark.parametrize("case", sorted(YSHFL))
def test_resident_2d_shuffled_y_faces(torch_cuda, case):
    name, over = YSHFL[case]
    cfg = W.config(name, **over)
    M0 = W.initial_field(cfg)
    Hg, _ = gpu_micro(torch_cuda, cfg, M0, 1, kernel_variant=2)
    pts = sorted(set([0, 1, cfg.n_points // 2, cfg.n_points - 1]))
    Hr = O.micro_batch(cfg, M0, points=pts)
    assert rel_err(Hg[:, pts], Hr) < TOL[1], (case, rel_err(Hg[:, pts], Hr))


@pytest.mark.parametrize("case", RESIDENT_2D)
def test_resident_2d_kernel_parity(torch_cuda, case):
    """The shared-memory-resident 2D FP32 kernel (kernel_variant 2) against the FP64 oracle."""
    name, over = SMALL[case]
    cfg = W.config(name, **over)
    if name == "c3_2d_uneven":
        cfg = cfg.replace(eps_field=None, box_n_field=None)
    M0 = W.initial_field(cfg)
    Hg, _ = gpu_micro(torch_cuda, cfg, M0, 1, kernel_variant=2)
    Hr = O.micro_batch(cfg, M0)
    assert rel_err(Hg, Hr) < TOL[1], (case, rel_err(Hg, Hr))


# Boxes too large for one CTA: split by rows over a thread-block cluster, with the
# halo rows exchanged through distributed shared memory (canvas instances with
# compile-time strides, and the instance with strides from the box).
CLUSTER = {
    "canvas_80_odd": ("c2_2d", dict(n_macro=(5, 5, 1), box_n=75, micro_steps=30)),
    "canvas_128": ("c5_sweep", dict(n_macro=(5, 5, 1), box_n=128, micro_steps=20)),
    "box_strides_140": ("c2_2d", dict(n_macro=(5, 5, 1), box_n=140, micro_steps=20)),
    "box_strides_order2_101": ("c2_2d", dict(n_macro=(5, 6, 1), box_n=101, micro_steps=24, stencil_order=2)),
    # the largest box the resident kernel holds: box strides over a cluster of 8 CTAs
    "box_strides_160_cluster8": ("c2_2d", dict(n_macro=(5, 5, 1), box_n=160, micro_steps=12)),
}


@pytest.mark.parametrize("case", sorted(CLUSTER))
def test_resident_2d_kernel_clusters(torch_cuda, case):
    name, over = CLUSTER[case]
    cfg = W.config(name, **over)
    M0 = W.initial_field(cfg)
    Hg, _ = gpu_micro(torch_cuda, cfg, M0, 1, kernel_variant=2)
    pts = [0, 7, cfg.n_points - 1]
    Hr = O.micro_batch(cfg, M0, points=pts)
    assert rel_err(Hg[:, pts], Hr) < TOL[1], (case, rel_err(Hg[:, pts], Hr))


# 3D boxes: each split by z-planes over a cluster (planes beyond a CTA's slab read from
# the neighbouring CTAs' shared memory), or held by one CTA when small: the z-column
# kernel for 27^3 to 32^3 boxes, the z-slab kernel for smaller ones and for tabulated
# coefficients.
RESIDENT_3D = {
    # the z-column kernel (boxes of 27^3 to 32^3, cluster size chosen by occupancy)
    "n32_cluster7": ("c4_3d", dict(n_macro=(5, 5, 5), box_n=32, micro_steps=20)),
    "n31_column_odd": ("c4_3d", dict(n_macro=(5, 5, 5), box_n=31, micro_steps=20)),
    "n28_column": ("c4_3d", dict(n_macro=(5, 6, 5), box_n=28, mu_over_eps=1.6, micro_steps=26)),
    # the z-slab kernel

    "n21_cluster3_odd": ("c4_3d", dict(n_macro=(5, 5, 6), box_n=21, mu_over_eps=0.9, micro_steps=24)),
    "n16_one_cta": ("c4_3d", dict(n_macro=(5, 6, 5), box_n=16, mu_over_eps=0.9, micro_steps=30)),
}


@pytest.mark.parametrize("case", sorted(RESIDENT_3D))
def test_resident_3d_kernel(torch_cuda, case):
    name, over = RESIDENT_3D[case]
    cfg = W.config(name, **over)
    M0 = W.initial_field(cfg)
    Hg, _ = gpu_micro(torch_cuda, cfg, M0, 1, kernel_variant=2)
    pts = [0, 11, cfg.n_points - 1]
    Hr = O.micro_batch(cfg, M0, points=pts)
    assert rel_err(Hg[:, pts], Hr) < TOL[1], (case, rel_err(Hg[:, pts], Hr))


# 2-row thread tiles (tile_rows = 2: twice the threads per slab of the 4-row tiles), which
# the plan autotuner may pick per box size: packs, a ragged box, and boxes on clusters of
# 3 and 5 CTAs.
TR2 = {
    "pack_n24": ("c2_2d", dict(n_macro=(8, 8, 1), box_n=24, micro_steps=40)),
    "ragged_n37": ("c2_2d", dict(n_macro=(6, 7, 1), box_n=37, micro_steps=24)),
    "pack_n48": ("c5_sweep", dict(n_macro=(6, 6, 1), box_n=48, micro_steps=30)),
    "cluster3_n64": ("c2_2d", dict(n_macro=(6, 6, 1), box_n=64, micro_steps=30)),
    "cluster5_n96": ("c5_sweep", dict(n_macro=(5, 5, 1), box_n=96, micro_steps=20, alpha_micro=0.1)),
}


@pytest.mark.parametrize("case", sorted(TR2))
def test_resident_2d_two_row_tiles(torch_cuda, case):
    name, over = TR2[case]
    cfg = W.config(name, **over).replace(tile_rows=2)
    M0 = W.initial_field(cfg)
    Hg, _ = gpu_micro(torch_cuda, cfg, M0, 1, kernel_variant=2)
    pts = sorted(set([0, cfg.n_points // 2, cfg.n_points - 1]))
    Hr = O.micro_batch(cfg, M0, points=pts)
    assert rel_err(Hg[:, pts], Hr) < TOL[1], (case, rel_err(Hg[:, pts], Hr))


def test_resident_2d_kernel_uneven_boxes(torch_cuda):
    cfg = _uneven_small()
    M0 = W.initial_field(cfg)
    Hg, info = gpu_micro(torch_cuda, cfg, M0, 1, kernel_variant=2)
    N = info["N"]
    pts = sorted(set([int(np.argmin(N)), int(np.argmax(N))] +
                     list(np.random.default_rng(2).choice(cfg.n_points, 10, replace=False))))
    Hr = O.micro_batch(cfg, M0, points=pts)
    assert rel_err(Hg[:, pts], Hr) < TOL[1]


def test_resident_2d_kernel_full_size_sampled(torch_cuda):
    cfg = W.config("c2_2d")
    M0 = W.initial_field(cfg)
    Hg, _ = gpu_micro(torch_cuda, cfg, M0, 1, kernel_variant=2)
    assert np.all(np.isfinite(Hg))
    pts = sorted(set([0, cfg.n_points - 1] + list(np.random.default_rng(3).choice(cfg.n_points, 4, replace=False))))
    Hr = O.micro_batch(cfg, M0, points=pts)
    assert rel_err(Hg[:, pts], Hr) < TOL[1]


def _parse_plan_report(text):
    """{N: (number of candidates timed, index kept)} from hmm_plan_report's lines."""
    out = {}
    for line in text.strip().splitlines():
        head, rest = line.split(":", 1)
        timed, kept = rest.rsplit("->", 1)
        out[int(head[2:])] = (timed.count(" ms"), int(kept))
    return out


@pytest.mark.parametrize("name,over", [("c3_2d_uneven", dict(n_macro=(8, 8, 1), micro_steps=12)),
                                        ("c2_2d", {})], ids=["uneven_small", "c2_full"])
def test_resident_plan_autotuner(torch_cuda, name, over):
    """hmm_init times every resident-kernel instance that holds a box size on a
    sample of its boxes and keeps the fastest; the tuned plan keeps parity."""
    from paper_2108_09463_gb300 import HMM
    cfg = W.config(name, **over)
    M0 = W.initial_field(cfg)
    h = HMM(cfg, precision=1, kernel_variant=2)
    rep = _parse_plan_report(h.plan_report())
    info = h.box_info()
    Hg = h.micro_batch(torch_cuda.from_numpy(M0).cuda()).cpu().numpy()
    h.close()
    assert rep, "no box size had two candidates"
    sizes = set(int(v) for v in info["N"])
    for N, (timed, kept) in rep.items():
        assert N in sizes and timed >= 2 and 1 <= kept <= timed, (N, timed, kept)
    N = info["N"]
    pts = sorted(set([int(np.argmin(N)), int(np.argmax(N)), cfg.n_points - 1] +
                     list(np.random.default_rng(5).choice(cfg.n_points, 4, replace=False))))
    Hr = O.micro_batch(cfg, M0, points=pts)
    assert rel_err(Hg[:, pts], Hr) < TOL[1]
    h64 = HMM(cfg.replace(n_macro=(6, 6, 1), eps_field=None, box_n_field=None), precision=0)
    assert h64.plan_report() == ""
    h64.close()


FULL = [("c2_2d", 0), ("c2_2d", 1), ("c3_2d_uneven", 1)]


@pytest.mark.parametrize("name,precision", FULL)
def test_full_size_sampled(torch_cuda, name, precision):
    cfg = W.config(name)
    M0 = W.initial_field(cfg)
    Hg, info = gpu_micro(torch_cuda, cfg, M0, precision)
    assert np.all(np.isfinite(Hg))
    N = info["N"]
    rng = np.random.default_rng(1)
    if precision == 0:
        pts = [0, int(rng.integers(cfg.n_points))]
    else:
        pts = sorted(set([0, cfg.n_points - 1, int(np.argmax(N)), int(np.argmin(N))] +
                         list(rng.choice(cfg.n_points, 2, replace=False))))
    _, Hr = reference(cfg, M0, precision, pts)
    assert rel_err(Hg[:, pts], Hr) < TOL[precision], name


MACRO = {
    "1d": ("c1_1d", dict(n_macro=(16, 1, 1), box_n=81, micro_steps=100), 5),
    "2d": ("c2_2d", dict(n_macro=(8, 8, 1), box_n=24, micro_steps=30), 4),
    # MPE (eq. h_mpe): one RK4P start-up step, then MPE steps
    "1d_mpe": ("c1_1d", dict(n_macro=(16, 1, 1), box_n=81, micro_steps=100, macro_stepper=1), 5),
    "2d_mpe": ("c2_2d", dict(n_macro=(8, 8, 1), box_n=24, micro_steps=30, macro_stepper=1), 4),
}


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32"])
@pytest.mark.parametrize("case", sorted(MACRO))
def test_macro_steps_parity(torch_cuda, case, precision):
    from paper_2108_09463_gb300 import HMM
    name, over, nsteps = MACRO[case]
    cfg = W.config(name, **over)
    M0 = W.initial_field(cfg)
    h = HMM(cfg, precision=precision)
    M = torch_cuda.from_numpy(M0).cuda()
    h.macro_step(M, nsteps)
    Mg = M.cpu().numpy()
    st = O.MacroStepper(cfg, M0, dt=h.macro_dt())
    assert abs(h.macro_dt() / O.macro_dt(cfg) - 1) < 1e-14
    hmax = np.linalg.norm(st.havg(M0), axis=0).max()
    for _ in range(nsteps):
        st.step()
    err = np.abs(Mg - st.M).max()
    # each macro step moves M by dt * O(|H_avg|) through at most 4 stages, so an
    # H_avg error within TOL (relative to max |H_avg|) bounds the M error by the
    # expression below; the FP64 oracle adds its own rounding floor.
    tol = TOL[precision] + (ORACLE_FP64_FLOOR if precision == 0 else 0.0)
    bound = 4 * nsteps * h.macro_dt() * tol * hmax + 1e-14
    assert err < bound, (err, bound)
    assert np.abs(np.linalg.norm(Mg, axis=0) - 1).max() < 1e-13
    h.close()


def test_restart_is_bit_identical(torch_cuda):
    from paper_2108_09463_gb300 import HMM
    cfg = W.config("c2_2d", n_macro=(8, 8, 1), box_n=24, micro_steps=20)
    M0 = torch_cuda.from_numpy(W.initial_field(cfg)).cuda()
    a = HMM(cfg, precision=1)
    Ma = M0.clone()
    a.macro_step(Ma, 10)
    b = HMM(cfg, precision=1)
    Mb = M0.clone()
    b.macro_step(Mb, 6)
    hist, j = b.get_state()
    Msave = Mb.clone()
    b.close()
    c = HMM(cfg, precision=1)
    c.set_state(hist, j)
    c.macro_step(Msave, 4)
    assert torch_cuda.equal(Ma, Msave)
    a.close()
    c.close()


def test_graph_replay_equals_single_steps(torch_cuda):
    from paper_2108_09463_gb300 import HMM
    cfg = W.config("c2_2d", n_macro=(8, 8, 1), box_n=24, micro_steps=20)
    M0 = torch_cuda.from_numpy(W.initial_field(cfg)).cuda()
    a, b = HMM(cfg, precision=1), HMM(cfg, precision=1)
    Ma, Mb = M0.clone(), M0.clone()
    a.macro_step(Ma, 5)
    for _ in range(5):
        b.macro_step(Mb, 1)
    assert torch_cuda.equal(Ma, Mb)


# Macro steps in waves (hmm_macro_step_wave): each micro problem is solved by the same
# kernel instance from the same M whichever wave holds it, so n_waves calls must give
# hmm_macro_step's M and history bit for bit.
WAVES = {
    "2d_resident": ("c2_2d", dict(n_macro=(8, 8, 1), box_n=24, micro_steps=20), 1, {}),
    "2d_uneven": ("c3_2d_uneven", dict(n_macro=(12, 12, 1), micro_steps=12), 1, {}),
    "2d_generic_fp64": ("c2_2d", dict(n_macro=(8, 8, 1), box_n=24, micro_steps=20), 0, {}),
    "3d_zcolumn": ("c4_3d", dict(n_macro=(6, 6, 6), micro_steps=6), 1, {}),
    "2d_flux_mpe": ("c2_2d", dict(n_macro=(8, 8, 1), box_n=24, micro_steps=20, model=1, macro_stepper=1), 1, {}),
}


@pytest.mark.gpu
@pytest.mark.parametrize("case", sorted(WAVES))
def test_macro_step_in_waves_equals_macro_step(torch_cuda, case):
    from paper_2108_09463_gb300 import HMM
    name, over, precision, _ = WAVES[case]
    cfg = W.config(name, **over)
    M0 = torch_cuda.from_numpy(W.initial_field(cfg)).cuda()
    a, b = HMM(cfg, precision=precision), HMM(cfg, precision=precision)
    Ma, Mb = M0.clone(), M0.clone()
    start = 1 if getattr(cfg, "macro_stepper", 0) == 1 else 2
    a.macro_step(Ma, start)
    b.macro_step(Mb, start)
    for n_waves in (1, 5, 7):
        a.macro_step(Ma, 1)
        for w in range(n_waves):
            before = Mb.clone()
            b.macro_step_wave(Mb, w, n_waves)
            if w < n_waves - 1:
                assert torch_cuda.equal(Mb, before)   # M changes only at the last wave
        assert torch_cuda.equal(Ma, Mb), n_waves
        ha, ja = a.get_state()
        hb, jb = b.get_state()
        assert ja == jb and torch_cuda.equal(ha, hb)
    a.close()
    b.close()


@pytest.mark.gpu
def test_macro_step_in_waves_refusals(torch_cuda):
    from paper_2108_09463_gb300 import HMM, HmmError
    cfg = W.config("c2_2d", n_macro=(8, 8, 1), box_n=24, micro_steps=10)
    M = torch_cuda.from_numpy(W.initial_field(cfg)).cuda()
    h = HMM(cfg, precision=1)
    with pytest.raises(HmmError, match="start-up"):          # no MPEA history yet
        h.macro_step_wave(M, 0, 2)
    h.macro_step(M, 2)
    for wave, n in ((1, 2), (0, 0), (2, 2), (0, 65)):         # out of order or out of range
        with pytest.raises(HmmError) as ei:
            h.macro_step_wave(M, wave, n)
        assert ei.value.status == 1
    h.macro_step_wave(M, 0, 3)
    with pytest.raises(HmmError, match="order"):
        h.macro_step_wave(M, 2, 3)                            # wave 1 skipped
    with pytest.raises(HmmError, match="order"):
        h.macro_step_wave(M.clone(), 1, 3)                    # another M
    h.macro_step_wave(M, 1, 3)
    h.micro_batch(M)                                          # abandons the step in progress
    with pytest.raises(HmmError, match="order"):
        h.macro_step_wave(M, 2, 3)
    _, j = h.get_state()
    assert j == 2
    for w in range(3):
        h.macro_step_wave(M, w, 3)
    assert h.get_state()[1] == 3
    h.close()


def test_host_entry_points(torch_cuda):
    from paper_2108_09463_gb300 import HMM
    cfg = W.config("c2_2d", n_macro=(8, 8, 1), box_n=24, micro_steps=20)
    M0 = W.initial_field(cfg)
    h = HMM(cfg, precision=1)
    Hd = h.micro_batch(torch_cuda.from_numpy(M0).cuda()).cpu().numpy()
    Hh = np.empty_like(M0)
    h.micro_batch_host(np.ascontiguousarray(M0), Hh)
    assert np.array_equal(Hd, Hh)
    Md = torch_cuda.from_numpy(M0).cuda()
    h2 = HMM(cfg, precision=1)
    h2.macro_step(Md, 3)
    Mh = M0.copy()
    h.macro_step_host(Mh, 3)
    assert np.array_equal(Md.cpu().numpy(), Mh)


def test_nonfinite_input_reported(torch_cuda):
    from paper_2108_09463_gb300 import HMM, HmmError
    cfg = W.config("c2_2d", n_macro=(8, 8, 1), box_n=24, micro_steps=10)
    M0 = W.initial_field(cfg)
    M0[:, 9] = np.nan
    h = HMM(cfg, precision=1)
    with pytest.raises(HmmError) as ei:
        h.micro_batch(torch_cuda.from_numpy(M0).cuda())
    assert ei.value.status == 6
    # the handle stays usable after the error
    M1 = W.initial_field(cfg)
    H = h.micro_batch(torch_cuda.from_numpy(M1).cuda())
    assert torch_cuda.isfinite(H).all()
