"""Autotune the kernel choices for the benchmark's workloads and write the cache.

Runs ct_autotune (the library's own tuner: it times the integration-scale
passes as FP32 stencils or on the tensor cores, the work-unit length, the
stencil block and the eigen stage's form on a seeded synthetic annulus) for
the shapes the workloads process, and stores each best choice in the tuning
cache that plans read at creation, keyed by the GPU's name:

  annulus512   512^3, sigma 2 / rho 6, masked, FP32 outputs, both forms
  stream2048   2048 x 2048 x 1024 in 256^3 chunks, sigma 2 / rho 8, masked, mixed, F16
  tera4096     4096 x 4096 x 2048 in 384^3 chunks, sigma 3 / rho 9, masked, mixed, U8Q / F16
  crops        the uneven crops' sizes (2^19 .. 2^25 voxels, x extents a multiple
               of 8, of 4 or neither) at every sigma / rho pair, both forms, F16

Usage: python -m paper_2508_07476_gb300.tune [--out PATH] [--only NAME]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_CACHE = os.path.join(HERE, "tuning", "tune_cache.json")


def _jobs(only=None):
    from . import _lib
    tilt = (math.sin(math.radians(10.0)), 0.0, math.cos(math.radians(10.0)))
    F32, F16, U8Q = _lib.CT_OUT_F32, _lib.CT_OUT_F16, _lib.CT_OUT_U8Q
    jobs = []
    if only in (None, "annulus512"):
        for prec in (_lib.CT_PREC_MIXED, _lib.CT_PREC_FP32):
            jobs.append(("annulus512", _lib.make_params(2.0, 6.0, (255.5, 255.5, 255.5), tilt, prec), (512, 512, 512),
                         None, True))
    if only in (None, "stream2048"):
        jobs.append(("stream2048", _lib.make_params(2.0, 8.0, (1023.5, 1023.5, 511.5), tilt, _lib.CT_PREC_MIXED,
                                                    F16, F16, F16), (2048, 2048, 1024), (256, 256, 256), True))
    if only in (None, "tera4096"):
        jobs.append(("tera4096", _lib.make_params(3.0, 9.0, (2047.5, 2047.5, 1023.5), tilt, _lib.CT_PREC_MIXED,
                                                  F32, U8Q, F16), (4096, 4096, 2048), (384, 384, 384), True))
    if only in (None, "crops"):
        # one cube-like volume per size class l (2^l voxels, +-1 class each) and x class, both forms
        for prec in (_lib.CT_PREC_MIXED, _lib.CT_PREC_FP32):
            for l in (19, 21, 23, 25):
                e = round((2 ** l) ** (1 / 3))
                for nx in (e - e % 8, e - e % 8 + 4, e - e % 8 + 1):
                    for sigma in (1.0, 1.5, 2.0, 3.0):
                        for rho in (2.0, 4.0, 6.0, 8.0):
                            p = _lib.make_params(sigma, rho, (nx / 2, e / 2, e / 2), (0.0, 0.0, 1.0), prec,
                                                 F16, F16, F16)
                            jobs.append((f"crop{nx}x{e}x{e}_s{sigma}_r{rho}_p{prec}", p, (nx, e, e), None, False))
    return jobs


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=DEFAULT_CACHE)
    ap.add_argument("--only", choices=["annulus512", "stream2048", "tera4096", "crops"], default=None)
    args = ap.parse_args(argv)
    import torch
    from . import _lib, build
    build.build()
    _lib.load()
    torch.cuda.set_device(0)
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    t0 = time.perf_counter()
    for name, p, dims, chunk, masked in _jobs(args.only):
        r = _lib.ct_autotune(p, dims, masked, args.out, chunk=chunk)
        print(json.dumps({"job": name, "dims": dims, "chunk": chunk, **r}), flush=True)
    print(json.dumps({"tuned_s": time.perf_counter() - t0, "cache": args.out}), file=sys.stderr)


if __name__ == "__main__":
    main()
