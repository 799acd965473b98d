"""A fixed workload for profilers: a few matvecs of one plan.

    python -m paper_2407_03608_gb300.profile_case --eps 1e-5 [--n 1000000] [--precision fp32] [--matvecs 4]
    python -m paper_2407_03608_gb300.profile_case --d 3 --eps 1e-5 [--n 2000000]

Builds the plan for one synthetic workload, runs ``--matvecs`` matvecs and prints the
plan sizes.  d = 2: half uniform, half in eight Gaussian clusters, Matern 3/2.  d = 3:
uniform in the unit cube, Matern 5/2.  It does nothing else, so an ncu launch filter
(``-k``, ``-s``, ``-c``) sees only the plan build and the matvec kernels.
"""
import argparse


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--eps", type=float, default=1e-5)
    ap.add_argument("--n", type=int, default=1_000_000)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--matvecs", type=int, default=4)
    ap.add_argument("--transform", type=int, default=0)
    ap.add_argument("--d", type=int, default=2, choices=[2, 3])
    args = ap.parse_args()
    import torch
    import gpinputs
    import paper_2407_03608_gb300 as gpn
    w = gpinputs.config_2d(args.n, 1.5) if args.d == 2 else gpinputs.config_3d(args.n)
    dev = torch.device("cuda", 0)
    prec = gpn.GP_FP32 if args.precision == "fp32" else gpn.GP_FP64
    plan = gpn.Plan(torch.from_numpy(w.points).to(dev), torch.from_numpy(w.s).to(dev),
                    torch.from_numpy(w.l).to(dev), nu=w.nu, eps=args.eps, precision=prec,
                    transform=args.transform)
    a = torch.from_numpy(w.alpha).to(dev)
    out = None
    for _ in range(args.matvecs):
        out = plan.matvec(a)
    torch.cuda.synchronize()
    i = plan.info
    print({k: i[k] for k in ("nf", "M", "n_sigma", "kernel_width", "tile", "transform")}, float(out.norm()))


if __name__ == "__main__":
    main()
