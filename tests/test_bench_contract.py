"""The native benchmark line carries every key of its contract.  The native
arm needs a GPU, so this reads bench.py's source on the CPU: the dict
literal assigned to ``line`` in ``main`` and the ``cpu_baseline`` entry added
after it."""
import ast
import os

from conftest import ROOT

TOP = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
       "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "gpu_launches",
       "clocks"}
ROOFLINE = {"bound", "achieved", "peak", "unit", "frac", "traffic"}
E2E = {"value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"}
CPU_BASELINE = {"value", "unit", "cores", "kind", "sample"}


def _main():
    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    return next(f for f in tree.body if isinstance(f, ast.FunctionDef) and f.name == "main")


def _keys(d):
    return {k.value for k in d.keys if isinstance(k, ast.Constant)}


def _sub(d, key):
    for k, v in zip(d.keys, d.values):
        if isinstance(k, ast.Constant) and k.value == key:
            return v
    raise KeyError(key)


def test_native_line_keys():
    main = _main()
    lines = [n.value for n in ast.walk(main) if isinstance(n, ast.Assign)
             and any(isinstance(t, ast.Name) and t.id == "line" for t in n.targets)]
    assert len(lines) == 1 and isinstance(lines[0], ast.Dict)
    line = lines[0]
    assert TOP <= _keys(line), TOP - _keys(line)
    assert ROOFLINE <= _keys(_sub(line, "roofline"))
    assert E2E <= _keys(_sub(line, "e2e"))
    assert "workload" in _keys(_sub(line, "config"))
    assert _sub(line, "data").value == "synthetic"
    assert _sub(line, "scaling").value == "weak"
    assert _sub(_sub(line, "roofline"), "bound").value == "hbm"
    # cpu_baseline is added to the line on rank 0
    adds = [n.value for n in ast.walk(main) if isinstance(n, ast.Assign)
            and any(isinstance(t, ast.Subscript) and isinstance(t.value, ast.Name)
                    and t.value.id == "line" and isinstance(t.slice, ast.Constant)
                    and t.slice.value == "cpu_baseline" for t in n.targets)]
    assert len(adds) == 1 and CPU_BASELINE <= _keys(adds[0])
    assert _sub(adds[0], "kind").value == "oracle"


def test_defaults_finish_quickly_and_warm_up():
    main = _main()
    defaults = {}
    for n in ast.walk(main):
        if isinstance(n, ast.Call) and getattr(n.func, "attr", "") == "add_argument":
            name = n.args[0].value
            for kw in n.keywords:
                if kw.arg == "default" and isinstance(kw.value, ast.Constant):
                    defaults[name] = kw.value.value
    assert defaults["--gpus"] == 1
    assert defaults["--warmup"] >= 3
    assert defaults["--impl"] == "native"
