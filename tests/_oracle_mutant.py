"""pytest plugin that plants one mistake in a Python module before the tests that pin it run
(CPU only; test infrastructure for tests/test_oracle_mutants.py and tests/test_host_mutants.py).

``ORACLE_MUTANT`` holds a JSON list ``[module, old, new]``: the module's source is executed again
in its own namespace with the single occurrence of ``old`` replaced by ``new``, and the oracle
modules already imported are reloaded so that names they took from it see the planted version.
Child processes the tests spawn import the module afresh and do not see the mistake.  Without
the variable the plugin does nothing.
"""
import importlib
import json
import os
import sys

import pytest


def pytest_configure(config):
    spec = os.environ.get("ORACLE_MUTANT")
    if not spec:
        return
    mod_name, old, new = json.loads(spec)
    mod = importlib.import_module(mod_name)
    with open(mod.__file__) as f:
        src = f.read()
    if src.count(old) != 1:
        raise pytest.UsageError(f"{mod_name}: the text to replace occurs {src.count(old)} times")
    exec(compile(src.replace(old, new), mod.__file__, "exec"), mod.__dict__)
    for name, other in list(sys.modules.items()):
        if name.startswith("oracle.") and name != mod_name and other is not None:
            importlib.reload(other)
