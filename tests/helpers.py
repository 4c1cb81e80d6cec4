"""Shared test helpers: norm-wise error metric and library loading."""
import numpy as np


def normwise(x, ref):
    """max_i |x_i - ref_i| / max_i |ref_i| (pointwise relative error is meaningless at phi = 0
    nodes and on 1e13 backgrounds next to 1e19 peaks)."""
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    scale = np.abs(ref).max()
    if scale == 0:
        return float(np.abs(x).max())
    return float(np.abs(x - ref).max() / scale)


def header_functions(path):
    """Names of the functions declared in a C header (int/const char* returning prototypes)."""
    import re
    src = open(path).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(\w+)\s*\(", src, flags=re.M)))
