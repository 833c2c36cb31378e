"""Every global name a function of the host-side Python modules refers to is defined at
module level or is a builtin (the GPU-only code paths of bench.py and the binding cannot
run here, so a missing import would otherwise first show on a GPU machine)."""
import builtins
import os
import symtable

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
MODULES = ["bench.py", "__graft_entry__.py", "paper_2301_12869_gb300/lbm.py", "paper_2301_12869_gb300/partition.py",
           "paper_2301_12869_gb300/inputs.py", "paper_2301_12869_gb300/_build.py"]


def _module_names(table):
    return {s.get_name() for s in table.get_symbols() if s.is_assigned() or s.is_imported() or s.is_namespace()}


def _global_refs(table, out):
    for child in table.get_children():
        if child.get_type() == "function":
            for s in child.get_symbols():
                if s.is_global() and s.is_referenced():
                    out.append((child.get_name(), s.get_name()))
        _global_refs(child, out)


@pytest.mark.parametrize("rel", MODULES)
def test_functions_refer_only_to_defined_globals(rel):
    path = os.path.join(ROOT, rel)
    table = symtable.symtable(open(path).read(), path, "exec")
    defined = _module_names(table) | set(dir(builtins)) | {"__file__", "__name__"}
    refs = []
    _global_refs(table, refs)
    missing = sorted({(f, n) for f, n in refs if n not in defined})
    assert not missing, missing
