"""Run one reconstruction configuration on the synthetic 1920x1080 quarter-
sampling frame a few times and print the per-run device time: a fixed
workload for profilers (ncu captures of one kernel) and quick comparisons.

    python -m paper_2202_13926_gb300.run_case --support 16 --repeat 3
    python -m paper_2202_13926_gb300.run_case --precision tc_bf16x3
"""
import argparse
import json


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--support", type=int, default=32, help="S = B + 2L (8, 16 or 32)")
    ap.add_argument("--block", type=int, default=4, help="B")
    ap.add_argument("--iters", type=int, default=100, help="K")
    ap.add_argument("--precision", default="fp32", help="fp32, fp64, tc_bf16x3 or tc_tf32")
    ap.add_argument("--update", default="single", help="single or conj_pair")
    ap.add_argument("--repeat", type=int, default=3)
    args = ap.parse_args(argv)

    import torch
    import __graft_entry__
    from paper_2202_13926_gb300 import fsr, synth
    __graft_entry__.build()
    img, mask = synth.fhd_quarter_case()
    dev = torch.device("cuda:0")
    d_img, d_mask = torch.from_numpy(img).to(dev), torch.from_numpy(mask).to(dev)
    d_out = torch.empty_like(d_img)
    params = fsr.make_params(block=args.block, border=(args.support - args.block) // 2, iters=args.iters,
                             precision=args.precision, update=args.update)
    ms = []
    with fsr.Handle(0) as h:
        for _ in range(args.repeat):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            fsr.fsr_reconstruct(h.ptr, d_img, d_mask, params, d_out)
            b.record()
            b.synchronize()
            ms.append(a.elapsed_time(b))
        h.check_status()
    print(json.dumps({"support": args.support, "block": args.block, "iters": args.iters,
                      "precision": args.precision, "update": args.update, "ms": ms}))


if __name__ == "__main__":
    main()
