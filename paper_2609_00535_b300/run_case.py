"""Run one workload for many steps through the C ABI and print KE_max as it decays.

  python -m paper_2609_00535_b300.run_case --case flat2d --steps 300000 --every 5000
  python -m paper_2609_00535_b300.run_case --case droplet2d --N 8 --ne 4 --cfl 0.2 ...
  python -m paper_2609_00535_b300.run_case --case capwall2d --theta 60 --steps 300000

Prints one JSON line per case: time step, wall time per step, and KE_max at
evenly spaced checkpoints (stops early on a non-finite state).
"""
import argparse
import json
import math
import time

from . import inputs, semlbm


CASES = ("flat2d", "cylinder2d", "sphere3d", "capwall2d", "droplet2d", "droplet3d")


def make(args):
    kw = {}
    if args.case == "flat2d":
        ne = (args.ne, args.ne) if args.ne else (8, 8)
        return inputs.flat_wall_2d(N=args.N or 4, ne=ne, theta=math.radians(args.theta),
                                   beta=args.beta or 1e-3, tau=args.tau or 0.5, cfl=args.cfl)
    if args.case == "cylinder2d":
        return inputs.cylinder_2d(theta=math.radians(args.theta), N=args.N or 6, cfl=args.cfl)
    if args.case == "sphere3d":
        ne = (args.ne,) * 3 if args.ne else (16, 16, 16)
        return inputs.sphere_3d(N=args.N or 5, ne=ne, theta=math.radians(args.theta), cfl=args.cfl)
    if args.case == "capwall2d":      # stiff flat-wall drop started at its equilibrium cap
        return inputs.cap_on_wall_2d(math.radians(args.theta), N=args.N or 4, ne=args.ne or 8,
                                     cfl=args.cfl)
    if args.case in ("droplet2d", "droplet3d"):
        dim = 2 if args.case == "droplet2d" else 3
        if args.beta:
            kw["beta"] = args.beta
        if args.tau:
            kw["tau"] = args.tau
        if args.Cn:
            kw["Cn"] = args.Cn
        return inputs.periodic_droplet(dim=dim, ne=args.ne or 4, N=args.N or 8, cfl=args.cfl, **kw)
    raise SystemExit("unknown case " + args.case)


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", default="flat2d")
    ap.add_argument("--steps", type=int, default=100000)
    ap.add_argument("--every", type=int, default=5000)
    ap.add_argument("--N", type=int, default=None)
    ap.add_argument("--ne", type=int, default=None)
    ap.add_argument("--theta", type=float, default=60.0, help="degrees")
    ap.add_argument("--beta", type=float, default=None)
    ap.add_argument("--tau", type=float, default=None)
    ap.add_argument("--cfl", type=float, default=0.4)
    ap.add_argument("--Cn", type=float, default=None, help="interface width / diameter (droplets)")
    ap.add_argument("--force-split", type=int, default=0,
                    help="force in F**: 0 c_s^2 grad rho - rho grad mu, 1 -rho grad mu")
    args = ap.parse_args(argv)
    if args.case not in CASES:
        ap.error("unknown case %s (one of %s)" % (args.case, ", ".join(CASES)))
    if args.force_split not in (0, 1):
        ap.error("--force-split must be 0 or 1")
    if args.steps <= 0 or args.every <= 0:
        ap.error("--steps and --every must be positive")
    return args


def main(argv=None):
    args = parse_args(argv)
    case = make(args)
    case.force_split = args.force_split
    s = semlbm.Solver.from_case(case)
    s.set_density(case.rho0)
    out, done = [], 0
    t0 = time.perf_counter()
    while done < args.steps:
        s.step(args.every)
        done += args.every
        d = s.diagnostics()
        out.append((done, d["ke_max"]))
        if d["status"] != 0 or not d["ke_max"] < 1.0:
            break
    wall = time.perf_counter() - t0
    # viscous time t_eta = eta D / gamma and La = gamma D / eta^2 (Sec. 3.3), with
    # eta = rho_l nu and nu = tau c_s^2 dt; D the drop diameter (or 2R)
    gamma = (case.rho_l - case.rho_v) ** 3 * math.sqrt(2 * case.kappa * case.beta) / 6
    eta = case.rho_l * case.tau * case.dt / 3.0
    D = 2 * case.extra.get("R", 0.25)
    print(json.dumps({"case": case.name, "nodes": case.nodes, "dt": case.dt, "tau": case.tau,
                      "force_split": case.force_split, "La": gamma * D / eta ** 2,
                      "T_over_t_eta": done * case.dt * gamma / (eta * D),
                      "steps": done, "us_per_step": 1e6 * wall / done,
                      "ke_max": ["%d:%.2e" % x for x in out[:: max(1, len(out) // 12)]]
                      + ["%d:%.2e" % out[-1]]}))
    s.close()


if __name__ == "__main__":
    main()
