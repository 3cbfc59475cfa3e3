"""Summaries of ncu CSV logs for profiles/ and the bench's `traffic` field.

    python profile_summary.py launches LOG.csv
        per-kernel launches, total device time and share from an
        `ncu --metrics gpu__time_duration.sum --csv --log-file LOG.csv` run
        (printed as a table).

    python profile_summary.py traffic LOG.csv KIND [KIND ...]
        DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch
        of each kernel kind (library kind name, e.g. front_small) from an
        `ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum --csv` run,
        written to profiles/traffic.json with the sha256 of the kernel source
        the capture was taken on; bench.py reports it as `roofline.traffic`
        only while that source is unchanged.

    python profile_summary.py expr-traffic LOG.csv
        DRAM bytes of one sparse-expression evaluation: the last evaluation's
        launches (k_expr_one .. k_expr_out*) of a `bench.py --workload lll`
        capture, written to profiles/traffic_expr.json with the sha256 of the
        expression runner's source; the lll bench reports it as
        `roofline.traffic` while that source is unchanged.

Kernel names are matched to library kinds by their `k_<name>` stem.
"""
import collections
import csv
import hashlib
import json
import os
import re
import sys

ROOT = os.path.dirname(os.path.abspath(__file__))
KERNEL_SOURCE = os.path.join(ROOT, "paper_2110_12865_gb300", "csrc", "ssco_kernels.cu")

# library kernel kind -> kernel function stems that implement it
KIND_STEMS = {
    "assemble": ["k_assemble"], "front_small": ["k_front_small"], "front_vec": ["k_front_vec"],
    "front_tiny": ["k_tiny_factor"], "big_init": ["k_big_init"], "big_kscatter": ["k_big_kscatter"],
    "big_potrf": ["k_big_potrf"], "big_trsm": ["k_big_trsm"], "big_update_tc": ["k_big_update_tc", "k_big_update_tcp"],
    "big_update": ["k_big_update", "k_big_update_f32"],
    "fwd_solve": ["k_fwd", "k_fwd_warp", "k_tiny_fwd", "k_fsplit_init", "k_fsplit_step", "k_fwd_cluster"],
    "bwd_solve": ["k_bwd", "k_bwd_warp", "k_tiny_bwd", "k_bsplit_init", "k_bsplit_step", "k_bwd_cluster"],
    "resid": ["k_resid"], "check": ["k_check"],
}


def read_rows(path):
    hdr, out = None, []
    for r in csv.reader(open(path)):
        if r and r[0] == "ID":
            hdr = r
            continue
        if hdr and len(r) == len(hdr):
            out.append(dict(zip(hdr, r)))
    return out


def stem(name):
    m = re.search(r"(k_[a-z_0-9]+?)(?:<|I[fd]|E|\(|$)", name)
    return m.group(1) if m else name[:40]


def value(d, unit_scale):
    return float(d["Metric Value"].replace(",", "")) * unit_scale.get(d["Metric Unit"], 1.0)


def launches(path):
    agg = collections.OrderedDict()
    for d in read_rows(path):
        if d.get("Metric Name") != "gpu__time_duration.sum":
            continue
        name = d["Kernel Name"]
        key = stem(name) + ("<float>" if ("IfE" in name or "<float>" in name) else
                            "<double>" if ("IdE" in name or "<double>" in name) else "")
        ns = value(d, {"nsecond": 1, "usecond": 1e3, "msecond": 1e6, "second": 1e9})
        a = agg.setdefault(key, [0, 0.0])
        a[0] += 1
        a[1] += ns
    tot = sum(a[1] for a in agg.values())
    print(f"{'kernel':32s} {'launches':>8s} {'total_ms':>10s} {'share':>7s}")
    for k, (n, ns) in sorted(agg.items(), key=lambda kv: -kv[1][1]):
        print(f"{k:32s} {n:8d} {ns / 1e6:10.3f} {ns / tot:7.3f}")
    print(f"{'TOTAL':32s} {sum(a[0] for a in agg.values()):8d} {tot / 1e6:10.3f}")


def traffic(path, kinds):
    per = collections.defaultdict(lambda: collections.defaultdict(float))
    for d in read_rows(path):
        if d.get("Metric Name") not in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            continue
        by = value(d, {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "KB": 1e3, "MB": 1e6, "GB": 1e9})
        per[(d["ID"], stem(d["Kernel Name"]))][d["Metric Name"]] += by
    sha = hashlib.sha256(open(KERNEL_SOURCE, "rb").read()).hexdigest()
    dst = os.path.join(ROOT, "profiles", "traffic.json")
    out = {"source_sha256": sha, "kernels": {}}
    try:  # merge with earlier captures of the same kernel source
        old = json.load(open(dst))
        if old.get("source_sha256") == sha:
            out = old
    except Exception:
        pass
    for kind in kinds:
        stems = set(KIND_STEMS[kind])
        vals = [v["dram__bytes_read.sum"] + v["dram__bytes_write.sum"] for (i, st), v in per.items() if st in stems]
        if vals:
            out["kernels"][kind] = {"launches": len(vals), "dram_bytes_per_launch": sum(vals) / len(vals),
                                    "capture": os.path.basename(path)}
    json.dump(out, open(dst, "w"), indent=1)
    print(json.dumps(out, indent=1))


EXPR_SOURCE = os.path.join(ROOT, "paper_2110_12865_gb300", "csrc", "ssco_expr_run.cu")


def expr_traffic(path):
    per = collections.OrderedDict()
    for d in read_rows(path):
        st = stem(d["Kernel Name"])
        if not st.startswith("k_expr") or d.get("Metric Name") not in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            continue
        per.setdefault((int(d["ID"]), st), 0.0)
        per[(int(d["ID"]), st)] += value(d, {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9})
    launches = list(per.items())
    starts = [i for i, ((_, st), _) in enumerate(launches) if st == "k_expr_one"]
    last = launches[starts[-1]:]
    out = {"source_sha256": hashlib.sha256(open(EXPR_SOURCE, "rb").read()).hexdigest(),
           "dram_bytes_per_evaluation": sum(b for _, b in last), "launches": [st for (_, st), _ in last],
           "capture": os.path.basename(path)}
    json.dump(out, open(os.path.join(ROOT, "profiles", "traffic_expr.json"), "w"), indent=1)
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    if sys.argv[1] == "launches":
        launches(sys.argv[2])
    elif sys.argv[1] == "traffic":
        traffic(sys.argv[2], sys.argv[3:])
    elif sys.argv[1] == "expr-traffic":
        expr_traffic(sys.argv[2])
    else:
        raise SystemExit(__doc__)
