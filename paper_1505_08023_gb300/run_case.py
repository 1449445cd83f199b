"""Run one case of the path once (for profiling or a quick check).

    python -m paper_1505_08023_gb300.run_case --n 128 --cg-steps 20 --mixed-steps 20

Builds the N x N x N problem through the C ABI (mesh, assembly, conversion to
--format), then runs, as asked: one stand-alone SpMV (--spmv), the fused FP64
CG for --cg-steps steps (tol 0, or to --tol when --cg-steps is 0), the
single-reduction CG for --sr-steps steps, and the mixed-precision
reliable-update solve for --mixed-steps FP32 steps; or, with
--stencil-steps, the matrix-free operator and CG; or, with --conv, one
stride-1 convolution of the warm-start network (tensor-core kernels with
TMA-staged BF16 input and with FP32 input, then the CUDA-core kernel); or, with
--wgrad, one layer's weight gradient (tensor-core kernel, then CUDA-core
kernel); or, with --batch, the batched solver on a seeded batch of meshes.  With
--drop-csr the CSR arrays are released after conversion (smaller footprint
for profiler captures that save and restore device memory).  Prints one line
per step taken.
"""
from __future__ import annotations

import argparse

import torch

from . import fe


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--format", choices=["csr", "sell", "bcrs3", "vbcrs"], default="bcrs3")
    ap.add_argument("--spmv", action="store_true")
    ap.add_argument("--cg-steps", type=int, default=20)
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--sr-steps", type=int, default=0,
                    help="steps of the single-reduction CG (tol 0); 0: skip")
    ap.add_argument("--mixed-steps", type=int, default=0)
    ap.add_argument("--mixed-values", choices=["f32", "bf16"], default="f32")
    ap.add_argument("--drop-csr", action="store_true")
    ap.add_argument("--batch", type=int, nargs=3, metavar=("COUNT", "LO", "HI"), default=None,
                    help="instead of one mesh: COUNT cubic meshes N ~ U{LO..HI} (PCG64 seed 0) with "
                         "random face data, --cg-steps steps of the batched solver (1 RHS per chunk)")
    ap.add_argument("--conv", type=int, nargs=3, metavar=("CIN", "COUT", "N"), default=None,
                    help="instead of the solver: one stride-1 conv of the warm-start network on an "
                         "N^3 grid, tensor-core kernel then CUDA-core kernel")
    ap.add_argument("--wgrad", nargs=4, metavar=("MODE", "CIN", "COUT", "N"), default=None,
                    help="instead of the solver: the weight gradient of one layer (s1, s2 or t2) on an "
                         "N^3 input grid, tensor-core kernel then CUDA-core kernel")
    ap.add_argument("--stencil-steps", type=int, default=None,
                    help="instead of the stored matrix: the matrix-free operator once, then this many "
                         "matrix-free CG steps (tol 0; 0: solve to --tol)")
    a = ap.parse_args()
    if a.stencil_steps is not None:
        run_stencil(a.n, a.stencil_steps, a.tol)
        return
    if a.conv is not None:
        run_conv(*a.conv)
        return
    if a.wgrad is not None:
        run_wgrad(a.wgrad[0], *map(int, a.wgrad[1:]))
        return
    if a.batch is not None:
        run_batch(*a.batch, fmt=a.format, steps=a.cg_steps)
        return

    s = fe.System(a.n).build()
    A = s.matrix(a.format, "f64")
    Alo = s.matrix(a.format, a.mixed_values) if a.mixed_steps > 0 else None
    if a.drop_csr and a.format not in ("csr", "vbcrs"):
        s.cols = s.vals = None
        s.coords = None
        torch.cuda.empty_cache()
    x = torch.zeros(s.m, dtype=torch.float64, device="cuda")
    if a.spmv:
        y = torch.empty_like(x)
        fe.fe_spmv(A.desc, s.b, y)
        print("spmv done")
    if a.cg_steps >= 0:
        tol, steps = (0.0, a.cg_steps) if a.cg_steps > 0 else (a.tol, 100000)
        r = fe.fe_cg_solve(A.desc, s.b, x, tol, steps, fe.cg_workspace(A), check=False)
        print(f"cg: status {r.status} steps {r.iterations} relres {r.relres:.3e}")
    if a.sr_steps > 0:
        x.zero_()
        r = fe.fe_cg_solve_sr(A.desc, s.b, x, 0.0, a.sr_steps, fe.sr_workspace(A), check=False)
        print(f"cg_sr: status {r.status} steps {r.iterations} relres {r.relres:.3e}")
    if Alo is not None:
        x.zero_()
        r = fe.fe_cg_solve_mixed(A.desc, Alo.desc, s.b, x, a.tol, fe.FE_MIXED_RELIABLE, 200, 0.1,
                                 a.mixed_steps, fe.mixed_workspace(Alo), check=False)
        print(f"mixed: status {r.status} fp32 steps {r.inner_iterations} "
              f"refinements {r.outer_iterations} relres {r.relres:.3e}")
    torch.cuda.synchronize()


def run_batch(count: int, lo: int, hi: int, fmt: str, steps: int):
    import fe_inputs
    sizes = [int(n) for n in fe_inputs.batched_sizes(0, count, lo=lo, hi=hi)]
    faces = [fe_inputs.face_data(0, i, n, n, n) for i, n in enumerate(sizes)]
    batch = fe.Batch(sizes, faces, fmt)
    plan = fe.fe_cg_batched_plan(batch.mats, batch.b, batch.x, 1, batch.workspace())
    fe.fe_cg_batched_launch(plan, 0.0, steps)
    st, res = fe.fe_cg_batched_results(plan)
    print(f"batched: {count} meshes, {sum((n + 1) ** 3 for n in sizes):,} rows, {steps} steps, "
          f"statuses {sorted(set(r.status for r in res))}")


def run_stencil(n: int, steps: int, tol: float):
    st = fe.StencilSystem(n).build()
    x = torch.zeros(st.m, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    st.spmv(st.b, y)
    print("matrix-free spmv done")
    tol, steps = (0.0, steps) if steps > 0 else (tol, 100000)
    r = st.solve(x, tol, steps, check=False)
    print(f"matrix-free cg: status {r.status} steps {r.iterations} relres {r.relres:.3e}")


def run_conv(cin: int, cout: int, n: int):
    dims = (n, n, n)
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.randn((cin,) + dims, device="cuda", generator=g)
    w = torch.randn(cin, 27, cout, device="cuda", generator=g) * 0.1
    w16 = torch.empty(cin * 27 * cout, dtype=torch.bfloat16, device="cuda")
    fe.fe_nn_pack_weights(w, cin, cout, 0, 0, w16)
    b = torch.zeros(cout, device="cuda")
    y = torch.empty((cout,) + dims, device="cuda")
    if cout in fe.TC_COUT:
        img = fe.mma_image(cin, cout)
        fe.fe_nn_pack_weights_mma(w16, cin, cout, img)
        x16 = fe.bf16i_buffer(cin, dims, "cuda")
        fe.fe_nn_to_bf16i(x, cin, dims, x16)
        fe.fe_nn_conv3d_tc_bf16i("s1", x16, cin, dims, img, b, y, cout, dims, 1)
        print(f"tensor-core conv (TMA-staged BF16 input) {cin}->{cout} on {n}^3 done, "
              f"wait flag {fe.fe_nn_tc_check()}")
        fe.fe_nn_conv3d_s1_tc(x, cin, dims, img, b, y, cout, 1)
        print(f"tensor-core conv (FP32 input) {cin}->{cout} on {n}^3 done, wait flag {fe.fe_nn_tc_check()}")
    fe.fe_nn_conv3d(fe.NN_MODES["s1"], x, cin, dims, w16, b, y, cout, dims, 1)
    torch.cuda.synchronize()
    print(f"CUDA-core conv {cin}->{cout} on {n}^3 done")


def run_wgrad(mode: str, cin: int, cout: int, n: int):
    din = (n, n, n)
    dout = din if mode == "s1" else (tuple((v - 1) // 2 + 1 for v in din) if mode == "s2"
                                     else tuple(2 * (v - 1) + 1 for v in din))
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.randn((cin,) + din, device="cuda", generator=g)
    dy = torch.randn((cout,) + dout, device="cuda", generator=g)
    dw = torch.empty((cin, 27, cout), device="cuda")
    M = fe.NN_MODES[mode]
    work = torch.empty(fe.fe_nn_wgrad_tc_workspace(M, cin, din, cout, dout) // 4 + 1, device="cuda")
    fe.fe_nn_conv3d_weight_grad_tc(M, x, cin, din, dy, cout, dout, dw, work)
    torch.cuda.synchronize()
    print(f"tensor-core weight gradient {mode} {cin}->{cout} on {n}^3 done, wait flag {fe.fe_nn_tc_check()}")
    if mode == "t2":
        need, _ = fe.fe_nn_corr_workspace(2, cin, din, cout)
    else:
        need, _ = fe.fe_nn_corr_workspace(1 if mode == "s1" else 2, cout, dout, cin)
    work = torch.empty(need // 4 + 1, device="cuda")
    fe.fe_nn_conv3d_weight_grad(M, x, cin, din, dy, cout, dout, dw, work)
    torch.cuda.synchronize()
    print(f"CUDA-core weight gradient {mode} {cin}->{cout} on {n}^3 done")


if __name__ == "__main__":
    main()
