"""Run a few MD steps of one synthetic workload inside a profiler range.

For kernel captures with an external profiler started with ranges off
(`ncu --profile-from-start off ...`): the handle is built, the launch shape is
fixed (``--tuning``) or autotuned, ``--warmup`` steps run outside the range,
then ``--steps`` steps run inside ``cudaProfilerStart/Stop``.  Without a
profiler the range calls do nothing and the script prints the mean step time.

    python -m paper_2010_01559_gb300.profile_case --workload 2to1 --steps 1
    python -m paper_2010_01559_gb300.profile_case --workload large --n 131072 \
        --tuning 512,1,2,8 --steps 2

Workloads: ``2to1`` (2:1 electrolyte, N = 8001, P = 200), ``large`` (1:1
electrolyte at density 0.064, alpha = 0.3, r_c = 5, P = 500, N from ``--n``),
``water`` (rigid 3-site point charges, ``--n`` molecules).
"""
import argparse
import json


def make_workload(name, n):
    from . import workloads
    if name == "2to1":
        return workloads.config_2to1_mixed()
    if name == "large":
        return workloads.config_large(n or (1 << 20))
    if name == "water":
        return workloads.config_water(n or 10000)
    raise ValueError(f"unknown workload {name!r}")


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--workload", default="2to1", choices=["2to1", "large", "water"])
    ap.add_argument("--n", type=int, default=0)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--tuning", default="", help="rho_chunk,force_split,real_split,real_seg "
                    "(0 = the library's choice); empty: autotune")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "f64"])
    ap.add_argument("--graph", action="store_true", help="replay the step as a CUDA graph")
    args = ap.parse_args(argv)

    import torch
    from . import RBE, params_from

    wl = make_workload(args.workload, args.n)
    h = RBE(params_from(wl.params, n_max=wl.n))
    dt = torch.float32 if args.precision == "mixed" else torch.float64
    pos = torch.from_numpy(wl.pos_q()).cuda().to(dt).contiguous()
    vel = torch.zeros((wl.n, 4), dtype=dt, device="cuda")
    vel[:, :3] = torch.from_numpy(wl.vel).cuda().to(dt)
    if args.tuning:
        h.set_tuning(*[int(v) for v in args.tuning.split(",")])
    elif args.precision == "mixed":
        h.autotune(pos)
    h.set_graph(args.graph)
    step = torch.zeros(1, dtype=torch.int64, device="cuda")
    h.step(pos, vel, args.warmup, step)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.profiler.start()
    e0.record()
    h.step(pos, vel, args.steps, step)
    e1.record()
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    print(json.dumps({"workload": wl.name, "N": wl.n, "tuning": list(h.get_tuning()),
                      "steps": args.steps, "ms_per_step": e0.elapsed_time(e1) / args.steps}))
    h.close()


if __name__ == "__main__":
    main()
