"""Build the CUDA library libsv_gb300.so in-tree (paper_1804_04797_gb300/_build/).

Every translation unit is compiled by nvcc for sm_103a only, in parallel, then linked
into one shared library with a C ABI (include/sv.h).  No CMake.
"""
import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, 'csrc')
OUT = os.path.join(HERE, '_build')
LIB = os.path.join(OUT, 'libsv_gb300.so')
ARCH = ['-gencode', 'arch=compute_103a,code=sm_103a']
FLAGS = ['-O3', '-lineinfo', '-std=c++17', '-Xcompiler', '-fPIC', '-Xcompiler', '-O2',
         '--expt-relaxed-constexpr', '-I', os.path.join(ROOT, 'include'), '-I', CSRC]


def nvcc():
    exe = shutil.which('nvcc') or '/usr/local/cuda/bin/nvcc'
    return exe


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, '*.cu')) + glob.glob(os.path.join(CSRC, '*.cpp')))


def _headers():
    return (glob.glob(os.path.join(CSRC, '*.h')) + glob.glob(os.path.join(CSRC, '*.cuh')) +
            glob.glob(os.path.join(ROOT, 'include', '*.h')))


def _stale(obj, src, hdr_time):
    return (not os.path.exists(obj) or os.path.getmtime(obj) < max(os.path.getmtime(src), hdr_time))


def build(verbose=False, extra=()):
    os.makedirs(OUT, exist_ok=True)
    srcs = _sources()
    hdr_time = max([os.path.getmtime(h) for h in _headers()] + [0])
    jobs = []
    objs = []
    for s in srcs:
        obj = os.path.join(OUT, os.path.basename(s) + '.o')
        objs.append(obj)
        if _stale(obj, s, hdr_time):
            cmd = [nvcc(), '-c', s, '-o', obj] + ARCH + FLAGS + list(extra)
            if s.endswith('.cpp'):
                cmd = [nvcc(), '-x', 'cu', '-c', s, '-o', obj] + ARCH + FLAGS + list(extra)
            jobs.append(cmd)
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        results = list(ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs))
    for cmd, r in zip(jobs, results):
        if verbose and r.stderr:
            print(r.stderr)
        if r.returncode != 0:
            raise RuntimeError('nvcc failed: %s\n%s%s' % (' '.join(cmd), r.stdout, r.stderr))
    if jobs or not os.path.exists(LIB):
        tmp = LIB + '.tmp%d' % os.getpid()
        cmd = [nvcc(), '-shared', '-o', tmp] + objs + ARCH + ['-lcuda']
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError('link failed: %s\n%s%s' % (' '.join(cmd), r.stdout, r.stderr))
        os.replace(tmp, LIB)
    return LIB


if __name__ == '__main__':
    import sys
    print(build(verbose='-v' in sys.argv))
