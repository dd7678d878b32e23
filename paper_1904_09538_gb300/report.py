"""Calibrated parameter values as rates (the conversions of the paper's
Table mm_param_vals, Section "Matrix Multiplication").

A parameter is a cost in seconds per counted unit.  A unit counted per
sub-group (granularity "SG") stands for the same work on all 32 of its
work-items; a unit counted per work-item ("WI") for one work-item's.  The
rate is the work per second: flops for arithmetic (a multiply-add is 2),
bytes for memory accesses."""

SUBGROUP = 32


def rate(param, granularity, per_work_item):
    """Work per second implied by a cost `param` (s per counted unit) of a
    feature counted at `granularity` ("SG" or "WI"), each work-item of a
    unit doing `per_work_item` flops or bytes."""
    if granularity not in ("SG", "WI"):
        raise ValueError("granularity must be 'SG' or 'WI'")
    if not param > 0:
        return None
    return (SUBGROUP if granularity == "SG" else 1) * per_work_item / param
