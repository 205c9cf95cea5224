"""bench.py runs one rank per GPU; every rank must enter the same collectives
in the same order, or the run hangs. Checked on the source (no GPU): no
function that reaches a collective (barrier, max/sum over ranks, the
whole-job rate, torch.distributed) is called under a condition on the rank."""
import ast
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TREE = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
PRIMITIVES = {"barrier", "reduce_over_ranks", "whole_job_rate"}


def _called_names(node):
    out = set()
    for n in ast.walk(node):
        if isinstance(n, ast.Call):
            f = n.func
            if isinstance(f, ast.Name):
                out.add(f.id)
            elif isinstance(f, ast.Attribute) and isinstance(f.value, ast.Name) and f.value.id == "dist":
                out.add("dist." + f.attr)
    return out


def collective_functions():
    funcs = {n.name: n for n in TREE.body if isinstance(n, ast.FunctionDef)}
    reach = set(PRIMITIVES)
    changed = True
    while changed:
        changed = False
        for name, fn in funcs.items():
            if name in reach:
                continue
            called = _called_names(fn)
            if called & reach or any(c.startswith("dist.") for c in called):
                reach.add(name)
                changed = True
    return reach - {"dist_setup", "main"}   # set-up and teardown run on every rank by construction


def _rank_conditions():
    for n in ast.walk(TREE):
        if isinstance(n, ast.If):
            names = {x.id for x in ast.walk(n.test) if isinstance(x, ast.Name)}
            if names & {"rank", "extras"}:
                yield n


def test_no_collective_under_a_rank_condition():
    coll = collective_functions()
    assert {"barrier", "reduce_over_ranks", "whole_job_rate", "timed", "e2e_leg"} <= coll
    bad = []
    for node in _rank_conditions():
        for part in node.body + node.orelse:
            hit = _called_names(part) & coll
            if hit:
                bad.append((node.lineno, sorted(hit)))
    assert not bad, bad


def test_the_check_sees_a_planted_collective():
    src = "def f(rank, ws):\n    if rank == 0:\n        x = reduce_over_ranks(1, ws, 'sum')\n"
    tree = ast.parse(src)
    node = next(n for n in ast.walk(tree) if isinstance(n, ast.If))
    assert _called_names(node.body[0]) & {"reduce_over_ranks"}
