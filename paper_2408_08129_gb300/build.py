"""Build the CUDA library in-tree with nvcc (sm_103a only).

Every translation unit under ``csrc/``, plus one generated unit per
(dimension, degree, precision) of the operator kernels, is compiled in
parallel into ``_build/`` and linked into ``_lib/libdgatmo.so``.  Recompiles
only sources newer than their object (headers count for every unit).
"""

import concurrent.futures
import glob
import os
import platform
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build", platform.machine())
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libdgatmo.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the DG library")


def _flags(src):
    common = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-lineinfo", ARCH, "-I", os.path.join(HERE, "..", "include")]
    if src.endswith(".cpp"):
        return common
    return common + ["--expt-relaxed-constexpr"]


# The operator kernels (ops_impl.cuh) are compiled once per (dimension, degree,
# precision), each in a translation unit of its own, so that the slowest part
# of the build spreads over all cores.
DIMS, DEGREES, PRECISIONS = (2, 3), (1, 2, 3, 4, 5), (("f64", "double"), ("f32", "float"))


def _generated_units():
    gen = os.path.join(BUILD, "gen")
    os.makedirs(gen, exist_ok=True)
    units = []
    for dim in DIMS:
        for deg in DEGREES:
            for tag, ctype in PRECISIONS:
                path = os.path.join(gen, "ops_%dd_r%d_%s.cu" % (dim, deg, tag))
                text = ('// generated by build.py: operator kernels for dim %d, degree %d, %s\n'
                        '#include "%s"\n\nnamespace dg {\nDG_INSTANTIATE_DEGREE(%d, %d, %s)\n}  // namespace dg\n'
                        % (dim, deg, ctype, os.path.join(CSRC, "ops_impl.cuh"), dim, deg, ctype))
                if not os.path.exists(path) or open(path).read() != text:
                    with open(path, "w") as f:
                        f.write(text)
                units.append(path)
    return units


def build(verbose=False, jobs=None):
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    sources = sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))
    sources += _generated_units()
    headers = glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(
        os.path.join(HERE, "..", "include", "*.h"))
    newest_header = max((os.path.getmtime(h) for h in headers), default=0.0)
    jobs_list = []
    objects = []
    for src in sources:
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        objects.append(obj)
        if os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(src), newest_header):
            continue
        jobs_list.append((src, obj))

    def compile_one(item):
        src, obj = item
        cmd = [nvcc] + _flags(src) + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("compile failed: %s\n%s\n%s" % (" ".join(cmd), r.stdout, r.stderr))
        if verbose:
            sys.stdout.write("compiled %s\n" % os.path.basename(src))
        return obj

    if jobs_list:
        n = jobs or min(len(jobs_list), os.cpu_count() or 4)
        # longest units first (the 3D operator kernels of high degree)
        jobs_list.sort(key=lambda it: (("ops_3d" in it[0]) * 10 + ("_r5" in it[0]) + ("_r4" in it[0])), reverse=True)
        with concurrent.futures.ThreadPoolExecutor(max_workers=n) as ex:
            list(ex.map(compile_one, jobs_list))
    if jobs_list or not os.path.exists(LIB):
        cmd = [nvcc, "-shared", ARCH, "-o", LIB + ".tmp"] + objects
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed: %s\n%s" % (r.stdout, r.stderr))
        os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
