"""Measures the maintenance cost model's lambda(s) on the current GPU (qk_profile_scan) and prints
one JSON object: {"d", "k", "metric", "sizes", "us": {storage: [microseconds per item]}}.

    python -m paper_2506_03437_b300.profile_lambda --d 128 --storage f32,bf16,fp8

The table goes to Index.maintain(lam_sizes=sizes, lam_us=us[storage], tau_us=...), tau in the
same unit (device microseconds per scanned (query, partition) item)."""

import argparse
import json

from . import _lib as L
from . import index

STORAGE = {"f32": L.STORE_F32, "bf16": L.STORE_BF16, "fp8": L.STORE_FP8}
METRIC = {"l2": L.METRIC_L2, "ip": L.METRIC_IP}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--d", type=int, default=128)
    ap.add_argument("--metric", choices=sorted(METRIC), default="l2")
    ap.add_argument("--storage", default="f32", help="comma-separated: f32, bf16, fp8")
    ap.add_argument("--sizes", default="16,64,256,1024,4096,16384,65536")
    ap.add_argument("--k", type=int, default=10)
    ap.add_argument("--reps", type=int, default=5)
    a = ap.parse_args(argv)
    sizes = [int(x) for x in a.sizes.split(",")]
    us = {}
    for st in a.storage.split(","):
        us[st] = index.profile_scan(a.d, sizes, k=a.k, reps=a.reps, metric=METRIC[a.metric],
                                    storage=STORAGE[st]).tolist()
    print(json.dumps({"d": a.d, "k": a.k, "metric": a.metric, "sizes": sizes, "us": us}))


if __name__ == "__main__":
    main()
