"""Host helpers of bench.py: the --impl pre-parse that pins the reference arm's BLAS to one
thread before numpy loads, and the worker count of the parallel oracle leg."""

import argparse
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_impl_argument_forms():
    b = load_bench()
    assert b._impl_arg(["bench.py", "--impl", "reference", "--steps", "2"]) == "reference"
    assert b._impl_arg(["bench.py", "--impl=reference"]) == "reference"
    assert b._impl_arg(["bench.py", "--steps", "2"]) is None
    assert b._impl_arg(["bench.py", "--impl"]) is None


def test_cpu_workers():
    b = load_bench()
    assert b.cpu_workers(argparse.Namespace(cpu_workers=0)) == 0
    assert b.cpu_workers(argparse.Namespace(cpu_workers=3)) == 3
    n = b.cpu_workers(argparse.Namespace(cpu_workers=-1))
    assert 1 <= n <= 64
