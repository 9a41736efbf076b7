"""Command-line runner: solves (or topology-optimises) one of the named
synthetic workloads through the C ABI and prints the statistics.

    python -m paper_1501_06211_gb300.run --workload c1 --solves 2
    python -m paper_1501_06211_gb300.run --workload c4 --topopt-steps 20 --learner history
    python -m paper_1501_06211_gb300.run --workload c4 --topopt-steps 40 --tol-eta 0.1
    python -m paper_1501_06211_gb300.run --workload c4 --topopt-steps 40 --tol-eta 0.1 \
        --learner history --coarse x0
    python -m paper_1501_06211_gb300.run --workload c1 --precision mixed --schur explicit \
        --theta 0.6 --relax-switch 1e-2 --relax-delta 0.2

Run from the repository root (the workload generators live in `workloads/`).
"""
import argparse
import json
import os
import sys


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--workload", default="c1", help="c0, c1, c2 or c4")
    ap.add_argument("--solves", type=int, default=1, help="solves of the assembled problem")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "mixed"])
    ap.add_argument("--schur", default="auto", choices=["implicit", "explicit", "auto"])
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--topopt-steps", type=int, default=0, help="Picard steps instead of solves")
    ap.add_argument("--learner", default="none", choices=["none", "history", "cnn", "cnn+history"])
    ap.add_argument("--tol-eta", type=float, default=0.0,
                    help="topology steps: adaptive tolerance from successive compliances (0: --tol)")
    ap.add_argument("--coarse", default="x0+correct", choices=["x0", "x0+correct"],
                    help="learner coarse space: Galerkin initial guess only, or with the correction")
    ap.add_argument("--sub", type=int, default=0,
                    help="subdomain edge in elements instead of the workload's own (0: keep)")
    ap.add_argument("--theta", type=float, default=0.5, help="theta of the face-local preconditioner")
    ap.add_argument("--relax-switch", type=float, default=0.0,
                    help="mixed precision: FP32 Schur complements once ||r|| <= this * ||f|| "
                         "(relaxed PCG with FP64 reliable updates; 0: refinement cycles)")
    ap.add_argument("--relax-delta", type=float, default=0.1,
                    help="relaxed PCG: residual drop between FP64 replacements")
    args = ap.parse_args(argv)
    sys.path.insert(0, os.getcwd())
    import torch
    import workloads
    from paper_1501_06211_gb300 import ddel

    cfg = workloads.config(args.workload)
    if args.sub > 0:
        cfg["sub"] = args.sub
    prec = {"fp64": ddel.DDEL_FP64, "fp32": ddel.DDEL_FP32, "mixed": ddel.DDEL_MIXED}[args.precision]
    mode = {"implicit": 0, "explicit": 1, "auto": 2}[args.schur]
    s = ddel.Solver(cfg, precision=prec, schur_mode=mode, tol=args.tol, max_it=20000, theta=args.theta,
                    relax_switch=args.relax_switch, relax_delta=args.relax_delta)
    if args.topopt_steps > 0:
        learner = None
        if args.learner != "none":
            m = {"history": ddel.DDEL_LEARN_HISTORY, "cnn": ddel.DDEL_LEARN_CNN,
                 "cnn+history": ddel.DDEL_LEARN_CNN_HISTORY}[args.learner]
            flags = ddel.DDEL_COARSE_X0 | (ddel.DDEL_COARSE_CORRECT if args.coarse == "x0+correct" else 0)
            learner = ddel.Learner(s, mode=m, k_history=4, coarse_flags=flags)
        ne = 1
        for n in cfg["ne"]:
            ne *= n
        vf = cfg.get("v_frac", 0.5)
        rho = torch.full((ne,), vf, dtype=torch.float64, device="cuda")
        ts = s.topopt_state(rho, vf, r_min=cfg.get("r_min", 1.5), learner=learner, tol_eta=args.tol_eta)
        for k in range(args.topopt_steps):
            st = s.topopt_step(ts)
            print(json.dumps({"step": k, "iters": st.iters, "coarse_k": st.coarse_k,
                              "compliance": ts.compliance, "change": ts.change,
                              "tol": ts.tol_used, "t_total_ms": st.t_total_ms}), flush=True)
        return
    s.assemble(workloads.density(cfg))
    s.factor()
    u = torch.zeros(s.n_dof, dtype=torch.float64, device="cuda")
    for k in range(args.solves):
        _, st = s.solve(None, u)
        print(json.dumps({"solve": k, **st.as_dict()}), flush=True)


if __name__ == "__main__":
    main()
