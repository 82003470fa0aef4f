/* LD_PRELOAD shim used by tests/test_abi_cpu.py: counts file-system calls
 * (open/openat/fopen/stat/access/dlopen families) made while armed, so a
 * test can show that run-time compilation opens no file.  Test support only. */
#define _GNU_SOURCE
#include <dlfcn.h>
#include <fcntl.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>
#include <sys/stat.h>

static volatile int armed = 0;
static volatile int count = 0;
static char log_buf[8192];
static int log_len = 0;

void shim_arm(int on) { armed = on; }
int shim_count(void) { return count; }
/* every call seen while armed, one "name path" per line */
const char *shim_log(void) { return log_buf; }

static void note(const char *what, const char *path) {
    if (!armed) return;
    __sync_fetch_and_add(&count, 1);
    if (log_len < (int)sizeof log_buf - 1)
        log_len += snprintf(log_buf + log_len, sizeof log_buf - log_len, "%s %s\n", what, path ? path : "(null)");
}

#define FWD(ret, name, params, args, pathexpr)               \
    ret name params {                                        \
        static ret(*real) params = 0;                        \
        if (!real) real = (ret(*) params)dlsym(RTLD_NEXT, #name); \
        note(#name, pathexpr);                               \
        return real args;                                    \
    }

int open(const char *p, int f, ...) {
    static int (*real)(const char *, int, ...) = 0;
    if (!real) real = (int (*)(const char *, int, ...))dlsym(RTLD_NEXT, "open");
    va_list ap; va_start(ap, f); int mode = va_arg(ap, int); va_end(ap);
    note("open", p);
    return real(p, f, mode);
}
int open64(const char *p, int f, ...) {
    static int (*real)(const char *, int, ...) = 0;
    if (!real) real = (int (*)(const char *, int, ...))dlsym(RTLD_NEXT, "open64");
    va_list ap; va_start(ap, f); int mode = va_arg(ap, int); va_end(ap);
    note("open64", p);
    return real(p, f, mode);
}
int openat(int d, const char *p, int f, ...) {
    static int (*real)(int, const char *, int, ...) = 0;
    if (!real) real = (int (*)(int, const char *, int, ...))dlsym(RTLD_NEXT, "openat");
    va_list ap; va_start(ap, f); int mode = va_arg(ap, int); va_end(ap);
    note("openat", p);
    return real(d, p, f, mode);
}
int openat64(int d, const char *p, int f, ...) {
    static int (*real)(int, const char *, int, ...) = 0;
    if (!real) real = (int (*)(int, const char *, int, ...))dlsym(RTLD_NEXT, "openat64");
    va_list ap; va_start(ap, f); int mode = va_arg(ap, int); va_end(ap);
    note("openat64", p);
    return real(d, p, f, mode);
}
FWD(FILE *, fopen, (const char *p, const char *m), (p, m), p)
FWD(FILE *, fopen64, (const char *p, const char *m), (p, m), p)
FWD(int, stat, (const char *p, struct stat *b), (p, b), p)
FWD(int, lstat, (const char *p, struct stat *b), (p, b), p)
FWD(int, access, (const char *p, int m), (p, m), p)
FWD(void *, dlopen, (const char *p, int f), (p, f), p)
