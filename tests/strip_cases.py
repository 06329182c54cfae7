"""Parity cases of the polyphase strip kernels, run in a child process with
FCFS_STRIP_KERNELS=1 (the kernels then take every 2D descriptor in their scope)
by tests/test_gpu_strip.py.  Each case compares the forward or the input
gradient with the FP64 oracle; the process exits non-zero on the first
failure and prints one line per case."""
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

NEAREST, BILINEAR, BICUBIC = 0, 1, 2

# (method, r, s, K for learnable taps or 0): the forward and adjoint window shapes the strip
# kernels are compiled for
SHAPES = [(BICUBIC, 2, 3, 0), (BICUBIC, 4, 3, 0), (BICUBIC, 3, 2, 0), (BICUBIC, 7, 5, 0), (BILINEAR, 3, 2, 0),
          (BILINEAR, 5, 4, 0), (BILINEAR, 5, 4, 2)]


def main():
    import oracle
    from paper_2203_10670_gb300 import build, fcfs, inputs

    assert os.environ.get("FCFS_STRIP_KERNELS") == "1"
    build.build()
    oracle.build()
    dev = torch.device("cuda", 0)
    ncase = 0
    for method, r, s, K in SHAPES:
        for dtype in (torch.float32, torch.bfloat16):
            for pad in (0, 1, 2):
                # ragged sizes: several strips (128 windows each) and bands, partial last strip
                shape = (2, 3, 97 + 11 * r, 8 * (60 + 7 * s))
                C = shape[1]
                if K:
                    g = torch.Generator().manual_seed(100 + r)
                    W, _ = fcfs.fcfs_make_weights(BILINEAR, r, s, K)
                    ws = [(torch.from_numpy(np.tile(W[None], (C, 1, 1))) + 0.05 * torch.randn((C,) + W.shape, generator=g))
                          .float().to(dev).contiguous() for _ in range(2)]
                    axes = [fcfs.Axis(r, s, method, K, w) for w in ws]
                    oax = [dict(r=r, s=s, K=K, w=w.double().cpu().numpy()) for w in ws]
                    poly = True
                else:
                    axes = [fcfs.Axis(r, s, method)] * 2
                    oax = [dict(r=r, s=s, method=method)] * 2
                    poly = False
                x = inputs.normal(shape, 7 + r, device=dev, dtype=dtype)
                y = fcfs.resize(x, axes, pad, 0.25)
                gy = inputs.normal(tuple(y.shape), 8 + r, device=dev, dtype=dtype)
                gx, _ = fcfs.resize_backward(None, gy, axes, pad, in_shape=shape, in_dtype=dtype)
                torch.cuda.synchronize()
                xh = x.double().cpu().numpy()
                gh = gy.double().cpu().numpy()
                want = oracle.resize(xh, oax, pad=pad, pad_value=0.25 if dtype == torch.float32 else
                                     float(torch.tensor(0.25, dtype=dtype)), polyphase=poly)
                tol = 2e-6 if dtype == torch.float32 else 1e-2
                ef = float(np.abs(y.double().cpu().numpy() - want).max()) / float(np.abs(xh).max())
                wdx = oracle.adjoint_dx(gh, shape[2:], oax, pad=pad)
                abs_ax = []
                for a in oax:
                    b = dict(a)
                    if "w" in a:
                        b["w"] = np.abs(a["w"])
                    else:
                        Wt, Kt = oracle.make_weights(a["method"], a["r"], a["s"])
                        b["w"], b["K"] = np.abs(Wt), Kt
                    abs_ax.append(b)
                scale = float(np.abs(gh).max())
                for a in abs_ax:
                    scale *= float(a["w"].sum(-1).max())
                edx = float(np.abs(gx.double().cpu().numpy() - wdx).max()) / scale
                ok = ef <= tol and edx <= tol
                print(f"{'ok' if ok else 'FAIL'} method={method} {r}/{s} K={K} {str(dtype)[6:]} pad={pad} "
                      f"fwd={ef:.2e} dx={edx:.2e}", flush=True)
                if not ok:
                    sys.exit(1)
                ncase += 1
    st = fcfs.fcfs_device_status(clear=True)
    print(f"cases={ncase} status={st}", flush=True)
    sys.exit(0 if st == 0 else 2)


if __name__ == "__main__":
    main()
