"""Autotuner for the sort and partition sweeps.

Every digit pass can run with one of ``configs()`` tile shapes (threads per block x
keys per thread, compiled into libbcf.so).  ``autotune()`` times each shape through
the C ABI on random keys of each requested size, keeps the fastest in the library's
host-side table (``bcf_tune_set``) and returns the choices; ``save()``/``load()``
keep the table in a text file keyed by device name and SM count (``bcf_tune_save``,
``bcf_tune_load``), so a process can load it at start-up instead of measuring again.  The inputs are random keys made
on the device with torch; they only exist to time the kernels.
"""
from __future__ import annotations

import ctypes
import os
import statistics

from . import OK, OP_PARTITION, OP_SEGMENTED_SORT, OP_SORT, BcfError, lib

OPS = {"sort": OP_SORT, "partition": OP_PARTITION, "segmented_sort": OP_SEGMENTED_SORT}


def configs():
    """[(threads, keys_per_thread)] of the compiled tile configurations."""
    L = lib()
    out = []
    for c in range(L.bcf_tune_num_configs()):
        t, k = ctypes.c_int(0), ctypes.c_int(0)
        if L.bcf_tune_config_info(c, ctypes.byref(t), ctypes.byref(k)) != OK:
            raise BcfError(1, "bcf_tune_config_info")
        out.append((t.value, k.value))
    return out


def candidates(op: str):
    """Configurations the table accepts for `op`: every one for the flat sort and
    partition; for the batched sort the 256 x 16 counts + scan forms (its plan
    cuts segments into 4096-key tiles)."""
    L = lib()
    if op != "segmented_sort":
        return list(range(L.bcf_tune_num_configs()))
    return [c for c, shape in enumerate(configs()) if shape == (256, 16) and L.bcf_tune_config_form(c) in (1, 2)]


def set_config(op: str, log2_n: int, config: int) -> None:
    rc = lib().bcf_tune_set(OPS[op], int(log2_n), int(config))
    if rc != OK:
        raise BcfError(rc, "bcf_tune_set")


def get_config(op: str, n: int) -> int:
    c = ctypes.c_int(0)
    rc = lib().bcf_tune_get(OPS[op], int(n), ctypes.byref(c))
    if rc != OK:
        raise BcfError(rc, "bcf_tune_get")
    return c.value


def _device_key():
    import torch
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return "%s/%dsm" % (p.name, p.multi_processor_count)


def _time(fn, reps, inner):
    """Median device time of one fn() call, in ms, from replays of a CUDA graph of
    `inner` calls: small inputs would otherwise time the host's launch cost."""
    import torch
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        for _ in range(2):
            fn()
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        for _ in range(inner):
            fn()
    g.replay()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        g.replay()
        b.record()
        b.synchronize()
        ts.append(a.elapsed_time(b) / inner)
    del g
    return statistics.median(ts)


def _workload(op, n, w):
    import torch

    from . import (partition, partition_workspace_size, segmented_sort, segmented_sort_workspace_size, sort,
                   sort_workspace_size, workspace)
    g = torch.Generator(device="cuda").manual_seed(0x150701391 + n)
    vals = torch.arange(n, dtype=torch.int32, device="cuda")
    ko, vo = torch.empty_like(vals), torch.empty_like(vals)
    if op == "segmented_sort":  # log-uniform segment sizes in [32, 2^18], n keys in all
        gc = torch.Generator().manual_seed(0x150701391 + n)
        sizes = []
        while sum(sizes) < n:
            sizes.append(int(2 ** (5 + 13 * torch.rand(1, generator=gc).item())))
        sizes[-1] -= sum(sizes) - n
        offs = torch.tensor([0] + sizes, dtype=torch.int64).cumsum(0).cuda()
        keys = torch.randint(-2**31, 2**31, (n,), dtype=torch.int32, device="cuda", generator=g)
        ws = workspace(segmented_sort_workspace_size(n, len(sizes), 4, 32))
        return lambda: segmented_sort(keys, vals, offs, keys_out=ko, vals_out=vo, ws=ws)
    if op == "sort":
        keys = torch.randint(-2**31, 2**31, (n,), dtype=torch.int32, device="cuda", generator=g)
        ws = workspace(sort_workspace_size(n, 4, 32))
        return lambda: sort(keys, vals, keys_out=ko, vals_out=vo, ws=ws)
    keys = (torch.randperm(n, device="cuda", generator=g) % w).to(torch.int32)
    ws = workspace(partition_workspace_size(n, w, 4, 1))
    return lambda: partition(keys, vals, w, balanced=True, keys_out=ko, vals_out=vo, ws=ws)


def autotune(ops=("sort", "partition"), log2_sizes=range(12, 27, 2), w=256, reps=5, verbose=False):
    """Time every configuration for each op and size 2^k, keep the fastest in the
    library's table and return {op: {k: (config, {config: ms})}}."""
    result = {}
    for op in ops:
        result[op] = {}
        for k in log2_sizes:
            n = 1 << k
            if op == "partition":
                n -= n % w
            fn = _workload(op, n, w)
            times = {}
            inner = max(1, min(32, (1 << 22) >> k))  # about 2^22 keys per replay
            for c in candidates(op):
                set_config(op, k, c)  # read at capture time: each config gets its own graph
                times[c] = _time(fn, reps, inner)
            best = min(times, key=times.get)
            set_config(op, k, best)
            result[op][k] = (best, times)
            if verbose:
                print("tune %-9s 2^%-2d -> config %d  %s" % (op, k, best,
                      " ".join("%d:%.4fms" % (c, t) for c, t in times.items())))
    return result


def cache_path():
    return os.environ.get("BCF_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "bcf", "tune.txt"))


def save(result=None, path=None):
    """Write the library's explicit table entries for this device to the cache
    file (bcf_tune_save; other devices' entries are kept).  `result` (from
    autotune) is accepted for convenience: its choices are already in the table."""
    path = path or cache_path()
    d = os.path.dirname(path)
    if d:
        os.makedirs(d, exist_ok=True)
    rc = lib().bcf_tune_save(path.encode())
    if rc != OK:
        raise BcfError(rc, "bcf_tune_save")
    return path


def load(path=None) -> bool:
    """Apply this device's cached entries (bcf_tune_load); returns whether any
    were found."""
    path = path or cache_path()
    if not os.path.exists(path):
        return False
    applied = ctypes.c_int(0)
    rc = lib().bcf_tune_load(path.encode(), ctypes.byref(applied))
    if rc != OK:
        raise BcfError(rc, "bcf_tune_load")
    return applied.value > 0
