"""Measured errors of the GPU tests, kept beside the pass/fail result."""
import os


def record(name, **values):
    """Append measured errors of a test (name and values, one JSON line) to the
    file named by the environment variable FDM_TEST_RECORD, if it is set: the
    margins of the parity bounds, kept beside the pass/fail result."""
    path = os.environ.get("FDM_TEST_RECORD")
    if not path:
        return
    import json
    with open(path, "a") as f:
        f.write(json.dumps({"test": name, **{k: float(v) for k, v in values.items()}}) + "\n")
