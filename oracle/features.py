"""Oracle: feature naming and model-feature matching (test infrastructure only).

Section "Kernel Features": a feature name starts with ``f_``; its first field
gives the class, the rest its characteristics.  Section "Data Motion
Features" fixes the field order of memory access features:

    f_mem_access_tag:<tag>_<mem type>_<data type>_<direction>_
        lstrides:{<constraints>}_gstrides:{<constraints>}_afr:<constraint>

every field optional.  Section "Gathering Kernel Statistics" fixes the count
granularity: arithmetic and local memory per sub-group, global memory per
work-item except lid(0)-stride-0 ("uniform") global accesses, which count per
sub-group; barriers are counted for a single work-item (Section
"Synchronization Features"); ``f_thread_groups`` is the work-group count and
``f_sync_kernel_launch`` is 1 (Sections "Synchronization Features", "Other
Features").
"""
from fractions import Fraction
import re

from . import raw_counts, dims

GRAN_WI, GRAN_SG, GRAN_WG, GRAN_K = "WI", "SG", "WG", "K"


def _afr_str(acc, foot):
    f = Fraction(int(acc), int(foot))
    return str(f.numerator) if f.denominator == 1 else "%d/%d" % (f.numerator, f.denominator)


def features(kernel, remove=None, **params):
    """Feature records of one kernel instance, from brute-force enumeration.

    Each record: name, count (at its granularity), gran, and for memory
    accesses the pattern fields (tag, mem, dtype, dir, lstr, gstr, afr).
    remove: global-access tags; the records are then those of the
    work-removed twin derived from this kernel's descriptor (Algorithm 3).
    """
    recs = raw_counts(kernel, remove=remove, **params)
    wdim, gdim = dims(kernel, params)
    out = []
    for r in recs:
        if r["kind"] == 0:
            out.append(dict(kind="op", name="f_op_%s_%s" % (r["dtype"], r["name"]), count=r["sg"],
                            count_wi=r["wi"], gran=GRAN_SG, dtype=r["dtype"], op=r["name"]))
        elif r["kind"] == 1:
            if not r["affine"]:
                raise ValueError("non-affine access %s in %s" % (r["name"], kernel))
            mem = "global" if r["mem"] == 0 else "local"
            d = "load" if r["dir"] == 0 else "store"
            ls = r["lstr"][:wdim]
            gs = r["gstr"][:gdim]
            uniform = mem == "global" and ls[0] == 0
            gran = GRAN_SG if (mem == "local" or uniform) else GRAN_WI
            name = "f_mem_access_tag:%s_%s_%s_%s_lstrides:{%s}_gstrides:{%s}_afr:%s" % (
                r["name"], mem, r["dtype"], d,
                ";".join("%d:%d" % (a, v) for a, v in enumerate(ls)),
                ";".join("%d:%d" % (a, v) for a, v in enumerate(gs)),
                _afr_str(r["wi"], r["footprint"]))
            out.append(dict(kind="mem", name=name, count=r["sg"] if gran == GRAN_SG else r["wi"], gran=gran,
                            tag=r["name"], mem=mem, dtype=r["dtype"], dir=d, dsize=r["dsize"], lstr=tuple(ls),
                            gstr=tuple(gs), loopstr=r["loopstr"], accesses=r["wi"], footprint=r["footprint"],
                            count_wi=r["wi"], count_sg=r["sg"]))
        elif r["kind"] == 2:
            if r["wi"] != r["sg"]:
                raise ValueError("work-items of %s see different barrier counts" % kernel)
            out.append(dict(kind="sync", name="f_sync_barrier_local", count=r["wi"], gran=GRAN_WI))
        elif r["kind"] == 3:
            out.append(dict(kind="groups", name="f_thread_groups", count=r["wi"], gran=GRAN_WG))
        elif r["kind"] == 4:
            out.append(dict(kind="launch", name="f_sync_kernel_launch", count=1, gran=GRAN_K))
        elif r["kind"] == 5:
            out.append(dict(kind="grid", name="grid", wg=r["lstr"], grid=r["gstr"]))
    return out


_CONS = re.compile(r"^(<=|>=|!=|<|>|=)?(-?[0-9]+(?:\.[0-9]+)?(?:/[0-9]+)?)$")


def _cons(text):
    m = _CONS.match(text)
    if not m:
        raise ValueError("bad constraint %r" % text)
    op = m.group(1) or "="
    val = Fraction(m.group(2))
    return op, val


def _ok(op, val, x):
    x = Fraction(x)
    return {"=": x == val, "!=": x != val, "<": x < val, ">": x > val, "<=": x <= val, ">=": x >= val}[op]


def _parse_strides(body):
    out = {}
    for part in body.split(";"):
        if not part:
            continue
        ax, c = part.split(":", 1)
        out[int(ax)] = _cons(c)
    return out


def parse_feature(name):
    """Parse a model feature name into a matcher description."""
    if name in ("f_sync_barrier_local", "f_thread_groups", "f_sync_kernel_launch"):
        return dict(kind={"f_sync_barrier_local": "sync", "f_thread_groups": "groups",
                          "f_sync_kernel_launch": "launch"}[name])
    if name.startswith("f_op_"):
        parts = name[len("f_op_"):].split("_")
        if len(parts) != 2 or parts[1] not in ("add", "mul", "madd"):
            raise ValueError("bad op feature %r" % name)
        return dict(kind="op", dtype=parts[0], op=parts[1])
    if name.startswith("f_mem_access"):
        rest = name[len("f_mem_access"):]
        d = dict(kind="mem")
        fields = [f for f in rest.split("_") if f]
        order = ["tag", "mem", "dtype", "dir", "lstrides", "gstrides", "afr"]
        pos = 0
        for f in fields:
            if f.startswith("tag:"):
                key, val = "tag", f[4:]
            elif f in ("global", "local"):
                key, val = "mem", f
            elif f in ("load", "store"):
                key, val = "dir", f
            elif re.match(r"^(float(32|64)(x[0-9]+)?|bfloat16)$", f):
                key, val = "dtype", f
            elif f.startswith("lstrides:{") and f.endswith("}"):
                key, val = "lstrides", _parse_strides(f[len("lstrides:{"):-1])
            elif f.startswith("gstrides:{") and f.endswith("}"):
                key, val = "gstrides", _parse_strides(f[len("gstrides:{"):-1])
            elif f.startswith("afr:"):
                key, val = "afr", _cons(f[4:])
            else:
                raise ValueError("bad field %r in %r" % (f, name))
            k = order.index(key)
            if k < pos:
                raise ValueError("field %r out of order in %r" % (f, name))
            pos = k + 1
            d[key] = val
        return d
    raise ValueError("unknown feature %r" % name)


def matches(desc, rec):
    if desc["kind"] != rec["kind"]:
        return False
    if desc["kind"] == "op":
        return rec["dtype"] == desc["dtype"] and rec["op"] == desc["op"]
    if desc["kind"] != "mem":
        return True
    for key in ("tag", "mem", "dtype", "dir"):
        if key in desc and rec[key] != desc[key]:
            return False
    for key, strides in (("lstrides", rec["lstr"]), ("gstrides", rec["gstr"])):
        for ax, (op, val) in desc.get(key, {}).items():
            if ax >= len(strides) or not _ok(op, val, strides[ax]):
                return False
    if "afr" in desc:
        op, val = desc["afr"]
        if not _ok(op, val, Fraction(int(rec["accesses"]), int(rec["footprint"]))):
            return False
    return True


def feature_value(name, recs):
    """Value of model feature `name` on a kernel's feature records: the sum of
    the counts (each at its own granularity) of all matching records."""
    desc = parse_feature(name)
    return sum(int(r["count"]) for r in recs if r["kind"] != "grid" and matches(desc, r))
