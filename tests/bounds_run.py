"""Run every streaming scheme, wavelet, storage type and direction at many
shapes through the library named by DWT2D_LIBRARY (the bounds-checked build)
and report any store the checks caught.  Started by test_gpu_bounds.py in a
process of its own; prints one line per failure and 'ok <n>' at the end."""
import sys

import numpy as np
import torch

from paper_1705_08266_gb300 import dwt2d as D
from paper_1705_08266_gb300 import synth

SHAPES = [(8, 8, 1), (8, 8, 3), (7, 9, 2), (9, 7, 3), (1, 9, 2), (9, 1, 2), (1, 1, 2), (2, 2, 1),
          (3, 3, 2), (33, 70, 3), (64, 300, 4), (130, 257, 5), (40, 513, 3), (65, 1000, 6),
          (301, 497, 4), (1030, 2050, 5), (777, 3001, 2), (16, 4099, 6), (4099, 16, 6)]


def main():
    bad = 0
    runs = 0
    for h, w, lv in SHAPES:
        for wavelet, dtypes in (("cdf97", (torch.float32, torch.float16)), ("legall53", (torch.int32,))):
            for dt in dtypes:
                x = synth.image(wavelet, h, w, h * 31 + w)
                if dt == torch.float16:
                    x = x / max(1.0, float(np.max(np.abs(x))))
                xd = D.empty_image(h, w, dt)
                xd.copy_(torch.from_numpy(x).to(dt))
                for scheme in ("separable", "nonsep", "nonsep_reduced"):
                    for fuse, cols in (("1", 2), ("2", 2), ("3", 4), ("1", 4), ("2", 4)):
                        if fuse == "3" and dt == torch.float16:
                            continue
                        opts = dict(fuse_max=int(fuse))
                        if cols == 4:
                            opts.update(fwd_cols_per_lane=4, inv_cols_per_lane=4)
                        plan = D.Plan(h, w, lv, wavelet, scheme, dt, options=opts)
                        ws = plan.workspace()
                        c = plan.forward(xd, workspace=ws)
                        plan.inverse(c, workspace=ws)
                        st = plan.status(ws)
                        runs += 1
                        if st != 0:
                            bad += 1
                            print(f"status {st}: {h}x{w} L{lv} {wavelet} {dt} {scheme} {opts}")
    # every shape in one batch, forward and inverse, in both batched forms and
    # at both tile widths
    jobs = []
    for i, (h, w, lv) in enumerate(SHAPES):
        for inv in (0, 1):
            x = torch.from_numpy(synth.image("cdf97", h, w, i)).to(torch.float32)
            src = D.empty_image(h, w, torch.float32)
            src.copy_(x)
            jobs.append((src, D.empty_image(h, w, torch.float32), lv, "cdf97", inv))
    for persistent in (0, 1):
        for cols in (2, 4):
            b = D.Batch(jobs, "nonsep_reduced", {"persistent": persistent, "cols_per_lane": cols})
            ws = b.workspace()
            b.upload(ws)
            b.launch(ws)
            st = b.status(ws)
            runs += 1
            if st != 0:
                bad += 1
                print(f"status {st}: batch persistent={persistent} cols={cols}")
    torch.cuda.synchronize()
    print(f"ok {runs}" if bad == 0 else f"failed {bad} of {runs}")
    return 1 if bad else 0


if __name__ == "__main__":
    sys.exit(main())
